/*
 * dsp.h — C ABI of the B300 GPU leaf-expansion library for HyP-DESPOT
 * (Cai, Luo, Hsu, Lee, "HyP-DESPOT: A Hybrid Parallel Algorithm for Online
 * Planning under Uncertainty", arXiv:1802.06215).
 *
 * The library runs the data-parallel part of the method, leaf-node
 * initialisation (Sec. III-D): for a batch of DESPOT leaves it steps the
 * deterministic model g(s, a, phi) for every (leaf, action, scenario)
 * (Eq. expand), groups each action's scenarios by observation into children
 * (Eq. newnodes), and initialises each child's upper bound from a heuristic
 * (Eq. ub) and its lower bound from default-policy rollouts to depth D
 * (Eq. lb), summed over the child's scenarios. Around it, a host tree search
 * with several CPU threads, scenario-based PO-UCT and virtual loss (Sec. III-C)
 * feeds leaves to the GPU.
 *
 * Conventions
 *  - Plain C: no C++ types or exceptions cross this boundary. Every call
 *    returns a dsp_status; dsp_last_error() gives the calling thread's last
 *    message.
 *  - Ownership: the caller allocates and frees every buffer passed in (device
 *    memory, or mapped pinned host memory where stated). The library owns only
 *    the opaque dsp_model, its constant tables and its small workspace.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Kernel calls are asynchronous on it unless stated otherwise.
 *  - State blocks: a scenario set is a uint32 array of `words` fields x
 *    `cap` scenarios, field-major (scenario i of field f at [f * cap + i]).
 *      Rock Sample (5 words): f0/f1 robot r as x | y<<8 | exited<<16 (f1 is 0
 *        with one robot), f2 good-rock mask, f3 sampled-rock mask, f4 scenario
 *        id.
 *      Car (4 + 2P + ceil(P/4) words): f0 distance s (float bits),
 *        f1 speed | terminal<<8, f2 scenario id, f3 zero, P words of
 *        pedestrian x, P of y (float bits), goals packed four per word.
 *  - Random numbers: phi_t of scenario id k is Philox4x32-10 (Salmon et al.,
 *    SC'11) at counter (k, t, purpose<<24 | element, plan_step) under key
 *    (seed low, seed high); the same under every action (Sec. III-A).
 *  - Observation keys are 64-bit; bit 62 marks a terminal outcome.
 *  - Sums over scenarios are int64 fixed point with scale 2^-32, each
 *    scenario's FP32 value rounded to nearest even before summing, so they are
 *    exact and independent of summation order.
 */
#ifndef DSP_H
#define DSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DSP_OK = 0,
  DSP_E_INVALID = 1,     /* bad argument; nothing was launched */
  DSP_E_OOM = 2,         /* an allocation of the library failed */
  DSP_E_CUDA = 3,        /* a CUDA runtime call failed (message has the name) */
  DSP_E_TIMEOUT = 4,     /* a bounded wait ran out (device or host side) */
  DSP_E_QUEUE_FULL = 5,  /* the device job queue has no free slot */
  DSP_E_UNSUPPORTED = 6, /* sizes beyond this build's limits */
  DSP_E_DEVICE = 7       /* a kernel reported an error in its status word */
} dsp_status;

typedef enum {
  DSP_MODEL_GRID = 0,      /* Rock Sample, one robot */
  DSP_MODEL_MULTIGRID = 1, /* Rock Sample, two robots */
  DSP_MODEL_CAR = 2,       /* car among pedestrians */
  DSP_MODEL_NAV = 3        /* navigation in a partially known map */
} dsp_model_kind;

typedef struct dsp_model dsp_model; /* opaque, owned by the library */

/* The POMDP (Sec. II-A: S, A, Z, T, O, R, gamma) of one task of Sec. IV-A,
 * with K scenarios and horizon D (Sec. III-A, Eq. lb). Caller-owned POD. */
typedef struct {
  int32_t kind;               /* dsp_model_kind */
  int32_t n;                  /* map side: Rock Sample 2..32, navigation 5..16 */
  int32_t m;                  /* Rock Sample rocks (1..32) */
  int32_t P;                  /* car: pedestrians (1..64) */
  float gamma;                /* discount */
  int32_t K;                  /* scenarios per planning step (1..512; one-robot Rock Sample 1..8192) */
  int32_t D;                  /* maximum depth (1..250) */
  uint64_t seed;              /* Philox key */
  uint32_t plan_step;         /* fourth Philox counter word */
  const int32_t* rock_cells;  /* host, m entries x | y<<8, distinct cells */
  float path_len, dt, ped_speed, sigma; /* car: path length, time step, walking speed, noise */
  double fail_p;              /* car: accelerate/decelerate fails; navigation: a move fails */
  double sense_p;             /* navigation: one adjacent-cell reading is wrong */
} dsp_model_desc;

/* Creates a model: validates the descriptor, builds its constant tables
 * (sensor thresholds floor((0.5 + 0.5 * 2^(-d/20)) * 2^32) by squared distance,
 * FP32 gamma^k, the 4096-entry inverse-normal table) on the host in FP64 and
 * uploads them to the current device. Returns DSP_E_INVALID on a bad
 * descriptor, DSP_E_CUDA/DSP_E_OOM on device failure; *out is NULL then. */
dsp_status dsp_create_model(const dsp_model_desc* desc, dsp_model** out);
void dsp_destroy_model(dsp_model* model);

int32_t dsp_state_words(const dsp_model* model);  /* words per scenario */
int32_t dsp_num_actions(const dsp_model* model);  /* |A| */
/* Max children per action the result arrays need (grid 4, multigrid 10,
 * navigation 257 (8-bit reading or terminal), car
 * n_scen). */
int32_t dsp_max_children(const dsp_model* model, int32_t n_scen);

/* Selects the random streams of a planning step (fourth counter word) for
 * every later call. */
dsp_status dsp_set_plan_step(dsp_model* model, uint32_t plan_step);

/* Copies a constant table to host memory for checks: which = 0 sensor
 * thresholds (uint64 per squared distance), 1 gamma^k (float, 256 entries),
 * 2 inverse-normal table (float, 4096). *count gets the entry count. */
dsp_status dsp_get_table(const dsp_model* model, int32_t which, void* host_out, int32_t* count);

/* Eq. expand for a batch: for each i < count,
 *   (out_i, obs_key[i], reward[i]) = g(in_i, actions[i], phi_depth).
 * in_block (cap in_cap), out_block (cap out_cap), actions, obs_key, reward:
 * device pointers. Scenarios already terminal stay put with reward 0. */
dsp_status dsp_step(const dsp_model* model, const uint32_t* in_block, int32_t in_cap, int32_t count,
                    const int32_t* actions, int32_t depth, uint32_t* out_block, int32_t out_cap,
                    uint64_t* obs_key, float* reward, void* stream);

/* Eq. lb for single scenarios: value[i] = sum_{t=start}^{D-1} gamma^(t-start) r_t
 * + gamma^(D-start) l(s_D) of the default policy rolled out from state i
 * (tail only if the horizon was reached alive). hist: device, 32 int8 belief
 * counters per scenario, or NULL for all zero. value: device float[count]. */
dsp_status dsp_rollout(const dsp_model* model, const uint32_t* block, int32_t cap, int32_t count,
                       const int8_t* hist, int32_t start_depth, float* value, void* stream);

/* One leaf expansion job (Sec. III-D, "MC_simulation": gather, update,
 * expansion, bounds). Every pointer is device memory (or mapped pinned host
 * memory). Result arrays are indexed by action a - first_action. */
typedef struct {
  const uint32_t* parent; /* state block holding the parent's scenario list */
  int32_t parent_cap;     /* its capacity (field stride) */
  int32_t n_scen;         /* |Phi_b|, 1..512; one-robot Rock Sample: up to 8192, above 512 only
                             with leaf_states (phase A keeps those leaves there, not in shared
                             memory); the device queue takes at most 512 */
  const uint16_t* idx;    /* n_scen positions of the leaf's scenarios in parent */
  int32_t last_action;    /* action into this leaf, applied at depth-1 ("update");
                             -1: parent already holds the leaf's states (a root) */
  int32_t depth;          /* depth of the leaf, 0..D-1 */
  int8_t hist[32];        /* belief counters of the leaf's history (per rock) */
  int32_t first_action, n_actions; /* actions [first, first + n) to expand */
  int32_t child_cap;      /* result capacity per action (dsp_max_children) */
  uint32_t* leaf_states;  /* out: the leaf's own states (cap n_scen), or NULL */
  int32_t* child_count;   /* out: [n_actions] children per action */
  int32_t* child_off;     /* out: [n_actions][child_cap + 1] offsets into perm */
  uint64_t* child_key;    /* out: [n_actions][child_cap] observation keys */
  int64_t* rew_sum;       /* out: [n_actions][child_cap] sum of step rewards */
  int64_t* u_sum;         /* out: [n_actions][child_cap] sum of u (Eq. ub) */
  int64_t* l_sum;         /* out: [n_actions][child_cap] sum of rollout values (Eq. lb) */
  uint16_t* perm;         /* out: [n_actions][n_scen] leaf positions grouped by child,
                             children in order of first occurrence, members in
                             position order */
} dsp_leaf_job;

/* Expands a batch of leaves in one persistent launch. `jobs` is a HOST array
 * of n_jobs descriptors (copied before return; the buffers it points to must
 * stay valid until the stream reaches the end of the work). Sums are
 * fixed point 2^-32. Validation failures return DSP_E_INVALID and launch
 * nothing; n_actions * child_cap >= 2^24 in a job, or more than 2^31
 * (action, scenario) pairs in the call, returns DSP_E_UNSUPPORTED. Asynchronous
 * on `stream`. Work buffers come from a memory pool the model owns: the job
 * table, the rollout-item list (Rock Sample: 20 B per (action, scenario) for
 * one robot, 24 B for two, 28 B and 32 B with a learned policy; navigation
 * 52 B) and, for Rock Sample's heuristic rollouts, the list of each child's
 * slices (32 B a slice, at most ceil(n_scen / 128) + 6 slices an action for
 * one robot, + 18 for two). The pool keeps its largest size mapped until
 * dsp_destroy_model, so repeated calls do not map memory again. */
dsp_status dsp_expand_leaves(dsp_model* model, const dsp_leaf_job* jobs, int32_t n_jobs, void* stream);

/* Device job queue (Sec. III-D, node-level parallelism: the paper launches one
 * kernel per leaf on the submitting thread's stream; here one persistent
 * kernel, launched from a CUDA graph, pulls leaf jobs that many host threads
 * submit). Jobs go into a ring of `capacity` slots in mapped pinned host
 * memory; the kernel takes them in ticket order, expands each (same results
 * as dsp_expand_leaves) and marks it done; it exits after idle_ns nanoseconds
 * without a job (0 = 2 ms) and a monitor thread relaunches it when jobs are
 * pending. Every model has its kernel: Rock Sample (a job's phase A on the
 * CTA that claims it, its rollout chunks shared by every CTA of the grid),
 * navigation (phase A and the job's rollouts on the claiming CTA) and the car
 * (the job's actions as units on the claiming CTA, lanes per scenario as the
 * expansion's default). Jobs of at most 512 scenarios (DSP_E_UNSUPPORTED
 * above); the kernels roll out the heuristic policy (DSP_E_UNSUPPORTED at
 * submit while a learned policy is set). All job pointers are device memory.
 * submit and wait are thread-safe. */
typedef struct dsp_queue dsp_queue;
dsp_status dsp_queue_create(dsp_model* model, int32_t capacity, uint64_t idle_ns, dsp_queue** out);
/* Publishes one job (copied, with the model's plan step at this moment: the
 * job draws its random streams under it); *ticket identifies it. A ring slot
 * is free again once its job has completed. Waits at most timeout_ns (0 = no
 * limit) for a free slot, else DSP_E_QUEUE_FULL with no ticket taken. */
dsp_status dsp_queue_submit(dsp_queue* queue, const dsp_leaf_job* job, uint64_t timeout_ns, uint64_t* ticket);
/* Waits at most timeout_ns (0 = no limit) until the job's results are written
 * (DSP_E_TIMEOUT otherwise); DSP_E_CUDA if the persistent kernel failed. */
dsp_status dsp_queue_wait(dsp_queue* queue, uint64_t ticket, uint64_t timeout_ns);
/* Kernel launches so far and tickets handed out. */
dsp_status dsp_queue_stats(dsp_queue* queue, uint64_t* launches, uint64_t* submitted);
/* Finishes the submitted jobs, stops the kernel and frees the queue. */
void dsp_queue_destroy(dsp_queue* queue);

/* Parameters of one planning step of the tree search (Sec. III-C). */
typedef struct {
  int32_t threads;       /* T search threads (trials per round), 1..256 */
  int32_t rounds;        /* trial budget: rounds (deterministic) or trials per thread (free running) */
  double time_limit_s;   /* free running: wall-clock budget, 0 = none */
  double c_a;            /* PO-UCT exploration scale (Eq. UCT); 0 = plain DESPOT argmax of the upper bound */
  double c_o;            /* virtual-loss scale, zeta = c_o * eps(b0) per traversing thread (Eq. augmented_WEU) */
  double xi;             /* target uncertainty ratio of WEU (Eq. select_lb) */
  double target_gap;     /* stop once the root gap U - L is at most this */
  int32_t deterministic; /* 1: rounds (select in thread order, one batched expansion, backups in thread order);
                            0: free-running threads, one CUDA stream each */
  int32_t use_queue;     /* free running: threads submit their leaves to one device job queue
                            (dsp_queue_*) instead of launching their own expansions; the model keeps that
                            queue (capacity max(64, 4 x threads)) until dsp_destroy_model */
  int32_t tree_lock;     /* free running: 0 = select and back up on per-node atomics without a lock (a leaf
                            claimed by compare-and-swap, counts as atomic increments, bounds as atomic stores;
                            the tree's bounds are recomputed bottom-up once the threads join); 1 = under
                            one tree lock */
  int32_t batch;         /* free running without the queue: > 1 = threads hand their claimed leaves to one
                            dispatching thread, which expands up to `batch` of them per dsp_expand_leaves
                            launch and backs them up; <= 1 = every thread launches its own leaf */
} dsp_search_params;

typedef struct {
  double root_u, root_l;     /* root bounds (weighted by |Phi_b0|/K) */
  int32_t action;            /* argmax_a of the lower bound of the root's actions, lowest index on ties */
  int32_t nodes, expansions, rounds;
  uint64_t scenario_steps;   /* g calls on live scenarios during the step */
  uint64_t signature;        /* digest of the tree in node-creation order (depth, key, bounds, |Phi|, visits) */
  double seconds;            /* wall-clock time of the step */
} dsp_search_result;

/* One planning step (Sec. III-A forward search, leaf initialisation on the
 * GPU, Eq. backup): builds a DESPOT tree over the n root scenarios (n <= K;
 * at most 512, or 8192 for one-robot Rock Sample without the device queue)
 * (root_states: HOST state block of capacity n; hist: HOST 32 belief
 * counters or NULL) with T threads, scenario-based PO-UCT for actions,
 * weighted excess uncertainty minus virtual loss for observations, one trial =
 * descend to one leaf, expand it, back up. Stops at the trial budget, the
 * time limit, a root gap <= target_gap, or when no branch is worth expanding.
 * Synchronous; root_visits (HOST, |A| entries, may be NULL) gets N(b0, a).
 * Device memory for the tree is allocated for the step and freed after it. */
dsp_status dsp_plan(dsp_model* model, const uint32_t* root_states, int32_t n, const int8_t* hist,
                    const dsp_search_params* params, dsp_search_result* result, int32_t* root_visits);

/* dsp_plan over several GPUs: node-level parallelism (Sec. III-D), the
 * paper's independent leaf expansions spread over devices. models: n_models
 * (1..64) models, one per GPU (each created with that GPU current), from the
 * same description, plan step and policy (DSP_E_INVALID otherwise). The
 * expansion with global index e of the step goes to models[e mod n_models]
 * (dsp_route_leaves); the new node's states and grouped positions stay on
 * that GPU, and a leaf whose parent's states live on another GPU first gets
 * them (and its scenario positions) by a peer copy on its own stream. The
 * model tables and the policy are replicated by construction (one model per
 * GPU); no kernel reads another GPU's memory; each expansion's small
 * results come back through host memory, which owns the tree. The root's
 * states go to models[0]. The device queue serves one model
 * (DSP_E_UNSUPPORTED with use_queue and n_models > 1, free running).
 * Deterministic rounds give the same tree as dsp_plan on one model, since an
 * expansion's results do not depend on the GPU that computes it. Results
 * and arguments otherwise as dsp_plan; scenario_steps sums all models. */
dsp_status dsp_plan_multi(dsp_model* const* models, int32_t n_models, const uint32_t* root_states, int32_t n,
                          const int8_t* hist, const dsp_search_params* params, dsp_search_result* result,
                          int32_t* root_visits);

/* The routing rule of dsp_plan_multi, on the host only (touches no GPU):
 * for n_leaves leaves that are expansions first_expansion, first_expansion
 * + 1, ... of a step, whose parents' states live on models parent_model[k]
 * (0..n_models-1), target[k] = (first_expansion + k) mod n_models and
 * copy[k] = 1 where target[k] != parent_model[k] (the parent's states and
 * the leaf's positions must be copied first), else 0. HOST arrays of
 * n_leaves entries. DSP_E_INVALID for bad arguments. */
dsp_status dsp_route_leaves(int32_t n_leaves, int64_t first_expansion, int32_t n_models, const int32_t* parent_model,
                            int32_t* target, int32_t* copy);

/* One node of a finished planning step, as dsp_plan_nodes exports it. */
typedef struct {
  int32_t depth;   /* tree depth, root 0 */
  int32_t n;       /* |Phi_b| */
  int32_t action;  /* argmax_a L(b, a), lowest index on ties: the action the tree's lower bound takes at b */
  int32_t visits;  /* N(b) */
  double U, L;     /* node bounds (weighted by |Phi_b|/K) */
  int8_t hist[32]; /* belief counters at b (per rock: sensed good minus sensed bad, clamped) */
} dsp_plan_node;

/* dsp_plan, then export of the tree (no counterpart in the paper; the source
 * of (state, action) pairs for imitation training of a learned default
 * policy): every expanded, non-terminal node with |Phi_b| >= min_scen, in
 * node-creation order, up to cap nodes. nodes: HOST array of cap records.
 * states: HOST state block of capacity cap (may be NULL) that receives the
 * first scenario of each exported node (position and sampled mask are common
 * to the node's scenarios in Rock Sample). *count = nodes written. */
dsp_status dsp_plan_nodes(dsp_model* model, const uint32_t* root_states, int32_t n, const int8_t* hist,
                          const dsp_search_params* params, dsp_search_result* result, int32_t* root_visits,
                          int32_t min_scen, int32_t cap, dsp_plan_node* nodes, uint32_t* states, int32_t* count);

/* POMCP-style planning (the single-scenario-per-path variant the paper names
 * among its future directions, Sec. V) on the same models and scenario
 * streams, with the GPU as the rollout service. UCT over histories: each
 * simulation carries one root scenario (simulation i of the plan takes
 * scenario i mod n) down the tree and rolls the default policy out from the
 * first new node. A round runs `batch` simulations level by level: at each
 * level the live simulations, in index order, choose by UCB1 on the action
 * values as they stood at the round's start plus one virtual visit per
 * earlier choice of the same action at the same node in this round (an
 * unvisited action first, lowest index on ties); one dsp_step call steps them
 * all; a simulation moves to the child of (action, observation), creating it
 * if new. It stops at a terminal outcome, at depth D (value 0 below), or at a
 * node created in this round, where it takes a rollout: one dsp_rollout call
 * per start depth. Backups run in simulation order: N += 1, N(a) += 1,
 * Q(a) += (G - Q(a)) / N(a) with G the discounted return. Nodes are numbered
 * in creation order (level, then simulation index).
 * root_states: HOST state block of n scenarios (capacity n). hist: HOST,
 * 32 counters (NULL = zeros). root_q / root_na: HOST arrays of |A| entries
 * (may be NULL). Planning stops after `rounds` rounds, or after time_limit_s
 * (> 0) at the end of a round. DSP_E_INVALID for bad arguments. */
typedef struct {
  int32_t rounds;       /* rounds of simulations, >= 1 */
  int32_t batch;        /* simulations per round, 1..65536 */
  double c;             /* UCB1 exploration constant */
  double time_limit_s;  /* 0 = none */
} dsp_pomcp_params;

typedef struct {
  int32_t action;           /* argmax_a Q(root, a) over visited actions, lowest index on ties */
  double value;             /* Q(root, action) */
  int32_t nodes, simulations, rollouts, rounds;
  uint64_t scenario_steps;  /* g calls on live scenarios (tree steps and rollouts) */
  uint64_t signature;       /* digest of the tree in creation order */
  double seconds;
} dsp_pomcp_result;

dsp_status dsp_pomcp_plan(dsp_model* model, const uint32_t* root_states, int32_t n, const int8_t* hist,
                          const dsp_pomcp_params* params, dsp_pomcp_result* result, double* root_q,
                          int32_t* root_na);

/* Launch shape of dsp_expand_leaves (the paper's fixed mapping of actions to
 * blocks and scenarios to threads, Sec. III-D, made a tunable): block = CTA
 * size of the Rock Sample rollout phase (128, 256 or 512; the car kernel runs
 * 256), tps = lanes sharing one car scenario (4, 8, 16 or 32; element-level
 * parallelism). 0 keeps the default (256; tps as dsp_set_launch_shape
 * states). Returns DSP_E_INVALID for other values. */
dsp_status dsp_set_tuning(dsp_model* model, int32_t block, int32_t tps);
dsp_status dsp_get_tuning(const dsp_model* model, int32_t* block, int32_t* tps);

/* The whole launch shape of dsp_expand_leaves (and of
 * dsp_expand_leaves_noalloc). The paper fixes the mapping of work to the GPU
 * (an action per thread block, a scenario per thread, factored elements per
 * warp; Sec. III-D); every field here is a measured choice instead. 0 keeps
 * each field's default.
 *  - block_b: rollout phase CTA size, Rock Sample (128, 256 or 512; default
 *    256): the scenarios (items) per CTA, one per thread.
 *  - ctas_b: rollout phase CTAs per SM, Rock Sample and navigation (1..32,
 *    capped by what fits; default as many as fit).
 *  - warps_a: Rock Sample grouping phase, warps per CTA (1..16): with A
 *    actions each warp expands about A / warps_a whole actions of a job
 *    (default: 5 warps with 12 or more jobs per SM for one robot, else up to
 *    16 warps of equal action counts).
 *  - tps: car, lanes sharing one scenario (4, 8, 16 or 32): the within-step
 *    split over pedestrians; with more pairs than lanes each lane takes
 *    ceil(pairs / tps) of them (the kernel is sized to that, up to four).
 *    Default: the tps whose pair slots (tps x pairs per lane) the crowd fills
 *    best, the largest on a tie (4 for 6 and 20 pedestrians, 8 for 12, 32
 *    for 50).
 *  - ctas_car: car kernel CTAs per SM (1..32, capped by what fits).
 *  - rs_form: one-robot Rock Sample with the heuristic default policy, how
 *    the grouping phase hands its (action, scenario) pairs to the rollout
 *    phase (dsp_expand_leaves only; the no-allocation entry point always
 *    uses items): 1 = blocks (the leaf's states, 12 B per scenario, and the
 *    grouped positions; the rollout phase rebuilds each pair's child state
 *    and mask: no per-pair list, about a seventh of the DRAM traffic),
 *    2 = items (a 20 B rollout item per pair, written by the grouping phase
 *    and read back; fewer instructions). Default 2.
 * One-robot Rock Sample has no within-step work to split (the default
 * policy reads one table entry per candidate rock), so its scenarios map one
 * to a thread. DSP_E_INVALID for values outside these sets. */
typedef struct {
  int32_t block_b, ctas_b, warps_a, tps, ctas_car, rs_form;
} dsp_launch_shape;
dsp_status dsp_set_launch_shape(dsp_model* model, const dsp_launch_shape* shape);
dsp_status dsp_get_launch_shape(const dsp_model* model, dsp_launch_shape* shape);

/* Autotuner over the launch shape: times dsp_expand_leaves on the caller's
 * jobs (HOST array; results are written to their buffers) for the default
 * shape and for every candidate of the model's kind, `reps` timed calls
 * each after one warm-up (CUDA events on `stream`), and keeps the fastest.
 *  - Rock Sample: block_b {128, 256, 512} x ctas_b {as many as fit, 6, 4} x
 *    warps_a {default, 5, 10} (two robots: {default, 8, 16}); one robot
 *    with the heuristic policy also x rs_form {blocks, items}.
 *  - car: tps {4, 8, 16, 32} x ctas_car {as many as fit, 3, 2}.
 *  - navigation: ctas_b {as many as fit, 6, 4, 2}.
 * best: the chosen shape (set in the model); best_ms / default_ms: mean time
 * per call of the chosen and the default shape; tried: candidates timed
 * (each may be NULL). Results of every call are identical whatever the
 * shape. */
dsp_status dsp_autotune_shape(dsp_model* model, const dsp_leaf_job* jobs, int32_t n_jobs, int32_t reps, void* stream,
                              dsp_launch_shape* best, float* best_ms, float* default_ms, int32_t* tried);

/* dsp_expand_leaves for callers that must not allocate device memory while
 * they plan (the paper has no counterpart). dsp_expand_leaves takes its work
 * buffers from the model's stream-ordered memory pool on every call; this entry point calls no
 * cudaMalloc, cudaFree or other allocating routine. It is for code that owns
 * all device memory through its own fixed pool, and for replanning loops with
 * a hard time budget, where an allocation call can block on the device.
 * Instead it runs the same Rock Sample kernels on one fixed scratch array that
 * the library keeps in device memory on every GPU that loads it (about 33 MB)
 * until the process exits.
 *  - Limits: Rock Sample models only (DSP_E_UNSUPPORTED for the car); at most
 *    8192 jobs and 2^20 (action, scenario) items (sum of n_scen * n_actions)
 *    per call. Larger calls fail with DSP_E_UNSUPPORTED and a message giving
 *    the limit; nothing is launched.
 *  - Set-up: the first call on a device looks up the array's device address
 *    with that device current. Make that first call before any stream capture
 *    on the device.
 *  - Sharing: every call uses the same array, which keeps the last call's
 *    contents; the counters the kernels need at zero are cleared on the
 *    stream at the start of each call. Calls that overlap on the GPU (other
 *    streams, other threads) race on the array: order them on one stream.
 *  - Host copies: `jobs` (a host array) is copied into one static host array
 *    of the library, page-locked once per process (it is pinned, not
 *    allocated), and from there to the device. So the call returns without
 *    waiting for earlier work on `stream`, except when the previous call's
 *    copy has not run yet: then it waits for that copy. If the system refuses
 *    to page-lock the array, the copy comes from pageable memory and the host
 *    may wait for the stream's earlier work.
 *  - Kernel timing (dsp_kernel_timing) creates events per call, so while it
 *    is on this entry point returns DSP_E_UNSUPPORTED.
 * Arguments, outputs, validation and the jobs' largest-first order are those
 * of dsp_expand_leaves. */
dsp_status dsp_expand_leaves_noalloc(dsp_model* model, const dsp_leaf_job* jobs, int32_t n_jobs, void* stream);

/* Learned default policy pi0 (the paper's pi0 is a hand-written default
 * policy, Sec. III-D, Eq. lb; this one is learned): an MLP 64 -> 256 -> 256 -> 32
 * with ReLU hidden layers whose first |A| logits score the actions and logit
 * |A| defers to the heuristic, trained with softmax cross-entropy on (state
 * features, action label) pairs (the shipped weights: approximate policy
 * iteration labels; planner imitation labels also work). FP32 master weights
 * with Adam; BF16 copies feed the tensor-core GEMMs (FP32 accumulation). Packed FP32 parameter layout (input-major):
 * W1[64][256] b1[256] W2[256][256] b2[256] W3[256][32] b3[32] (90656 floats).
 * Features of one-robot Rock Sample: x/n, y/n, then per rock (rock x - x)/n,
 * (rock y - y)/n, clamp(counter, -3, 3)/3, sampled; zero-padded to 64. */
typedef struct dsp_mlp dsp_mlp;
/* He-normal weights from `seed`, zero biases; buffers for batches <= max_batch. */
dsp_status dsp_mlp_create(int32_t max_batch, uint64_t seed, dsp_mlp** out);
void dsp_mlp_destroy(dsp_mlp* mlp);
dsp_status dsp_mlp_set_weights(dsp_mlp* mlp, const float* host_params);  /* packed FP32, host */
dsp_status dsp_mlp_get_weights(const dsp_mlp* mlp, float* host_params);
/* logits (device, B x 32 FP32) of features X (device, B x 64 FP32). */
dsp_status dsp_mlp_forward(dsp_mlp* mlp, const float* X, int32_t B, float* logits, void* stream);
/* Mean loss over the batch and its packed FP32 gradient (host), no update. */
dsp_status dsp_mlp_grad(dsp_mlp* mlp, const float* X, const int32_t* y, int32_t B, int32_t n_actions, float* loss,
                        float* grad_host, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr); *loss (host,
 * may be NULL) gets the batch's mean loss before the step. */
dsp_status dsp_mlp_train_step(dsp_mlp* mlp, const float* X, const int32_t* y, int32_t B, int32_t n_actions,
                              float lr, float* loss, void* stream);

/* Makes `mlp` (its current weights, copied) the default policy of every later
 * rollout of the model (dsp_expand_leaves, dsp_expand_leaves_noalloc,
 * dsp_rollout). At each rollout step the network maps the scenario's features
 * (dsp_features) to logits. The action is the argmax, lowest index on ties,
 * over the allowed actions and logit |A| ("defer", which takes the heuristic
 * policy's action).
 *  - Rock Sample: no move off the N, S or W border and no Sample off an
 *    unsampled rock; no Sense of a sampled rock or of one whose counter reads
 *    +-3.
 *  - Car: every action is allowed.
 * The network runs as tcgen05 tensor-core tiles over 128 live scenarios per
 * CTA, BF16 inputs with FP32 accumulation. g is still stepped exactly, so the
 * rollout value is a true policy value and l0 a valid lower bound. NULL
 * restores the heuristic policy. One-robot Rock Sample with at most 15 rocks,
 * or the car (DSP_E_UNSUPPORTED for two robots); the device job queue keeps
 * the heuristic policy. */
dsp_status dsp_set_policy(dsp_model* model, const dsp_mlp* mlp);
/* dsp_rollout with the learned policy, also recording every step's action
 * and the network's output that chose it:
 *  - actions (device, count x D int32, may be NULL) gets at
 *    [i * D + (t - start_depth)] the action taken at depth t;
 *  - logits (device, count x D x 32 FP32, 16-byte aligned, may be NULL) gets
 *    at [(i * D + (t - start_depth)) * 32 + c] logit c of that step as the
 *    tensor-core tile computed it (FP32 accumulator + bias), all 32 columns,
 *    before the allowed-action mask.
 * Entries of steps after a rollout ended are left as they were. */
dsp_status dsp_rollout_logged(const dsp_model* model, const uint32_t* block, int32_t cap, int32_t count,
                              const int8_t* hist, int32_t start_depth, float* value, int32_t* actions,
                              float* logits, void* stream);

/* The hand-written default policy pi0 of the model's rollouts (Sec. III-D,
 * Eq. lb) per state, and the learned policy's allowed actions, on the GPU,
 * so that training code labels states with the very functions the rollouts
 * run. block: device state block of capacity cap; hist: device count x 32
 * belief counters (Rock Sample; navigation: counter 0 holds the last
 * reading; may be NULL for the car); actions (device, count int32) gets the
 * action (two robots: the joint action a0 * (5 + m) + a1); allowed (device,
 * count uint32, may be NULL; one-robot Rock Sample only, DSP_E_UNSUPPORTED
 * otherwise) gets bit a set for every action the learned policy may take
 * and bit |A| (defer). Asynchronous on `stream`. */
dsp_status dsp_default_policy(const dsp_model* model, const uint32_t* block, int32_t cap, int32_t count,
                              const int8_t* hist, int32_t* actions, uint32_t* allowed, void* stream);

/* Policy features (the learned policy's input, the same function the learned
 * rollout evaluates): out (device, count x 64 FP32, 16-byte aligned); block:
 * device state block of capacity cap.
 *  - One-robot Rock Sample: row i = x/n, y/n, then per rock (rock x - x)/n,
 *    (rock y - y)/n, clamp(counter, -3, 3)/3, sampled, zero-padded. hist:
 *    device count x 32 counters.
 *  - Car: s / path length, v / 3, then for the 8 pedestrians nearest to the
 *    car (squared distance, lower index on ties) dx / 10, dy / 10 and 1 if the
 *    pedestrian is in the heuristic policy's danger zone (0 < dx <= 4,
 *    |dy| <= 1), zero-padded. hist is ignored (may be NULL). */
dsp_status dsp_features(const dsp_model* model, const uint32_t* block, int32_t cap, int32_t count,
                        const int8_t* hist, float* out, void* stream);

/* Measurement support (no counterpart in the paper): returns the summed GPU
 * time of the expansion kernels of every dsp_expand_leaves call recorded since
 * the last call (CUDA events on each call's stream, around its kernels only),
 * then turns recording on (enable = 1) or off. Synchronises those events. */
dsp_status dsp_kernel_timing(dsp_model* model, int32_t enable, double* total_ms, int32_t* calls);

/* Autotuner (the paper fixes the work-to-thread mapping, Sec. III-D; here it
 * is measured): times dsp_expand_leaves on the caller's jobs (HOST array, as
 * for dsp_expand_leaves; results are written to their buffers) for every
 * candidate launch shape, `reps` timed calls each after one warm-up, keeps the
 * fastest in the model (dsp_set_tuning) and returns it with its mean time in
 * ms. Synchronises `stream`. */
dsp_status dsp_autotune(dsp_model* model, const dsp_leaf_job* jobs, int32_t n_jobs, int32_t reps, void* stream,
                        int32_t* best_block, int32_t* best_tps, float* best_ms);

/* Scenario-steps (g calls on live scenarios: update + expansion + rollout
 * steps) counted by the kernels since the last reset, and the device status
 * word (0 = fine). Synchronises the device. */
dsp_status dsp_read_counters(dsp_model* model, uint64_t* scenario_steps, uint32_t* device_status);
dsp_status dsp_reset_counters(dsp_model* model, void* stream);

/* Measurement support (no counterpart in the paper): launches a kernel of
 * independent 32-bit integer xor/add chains over 8 CTAs of 256 threads per SM
 * and returns the integer operations it performs; the caller times it to get
 * the device's integer issue rate. sink: device, one uint32. */
dsp_status dsp_alu_probe(uint32_t* sink, int32_t iters, double* ops_per_launch, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* dsp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DSP_H */
