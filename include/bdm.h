/*
 * bdm.h -- C ABI of libbdm.so, the GB300 (sm_103a) agent-mechanics hot path of the BioDynaMo
 * simulation loop (Breitwieser et al., arXiv 2006.06775).
 *
 * The calls follow the paper's statement of a simulation (Sec. "Simulation concepts", Fig. 1D):
 * initialisation (bdm_create, bdm_add_agents, bdm_set_grid: place agents, set attributes, choose
 * behaviours), execution (bdm_step: agent operations -- behaviours and mechanical forces -- for every
 * agent each step, plus the standalone diffusion operation; bdm_diffusion_step: the standalone
 * operation alone), and read-out (bdm_get_state, including the SIR counting operation of Sec.
 * "Epidemiology use case").
 *
 * Conventions
 *  - Every function returns a bdm_status; 0 is success, negative is an error. bdm_last_error gives
 *    a message for the handle (thread-unsafe: one handle per host thread).
 *  - Ownership: the library owns the opaque handles and all device memory they hold. The caller owns
 *    every buffer it passes. Input pointers in this header are HOST pointers, copied in before the
 *    call returns; output pointers are HOST pointers filled before the call returns.
 *  - Ordering: state crosses the boundary in agent-id order (ids 0..n-1 in insertion order, then
 *    division daughters). Internally, mechanics agents live in box order on the device; SIR
 *    agents stay in id order with a box-order index.
 *  - Streams: work is enqueued on bdm_params.stream (a cudaStream_t; NULL = a non-blocking stream
 *    the handle creates and destroys) and is asynchronous, except bdm_get_state, which
 *    synchronises that stream. A device error word (grid overflow, capacity overflow, a bounded
 *    wait that timed out) is checked at the next synchronising call and returned as BDM_ESTATE /
 *    BDM_ENOMEM / BDM_ETIMEOUT; the handle then refuses further steps.
 *  - Memory: if alloc/free are given, every device allocation goes through them (for example the
 *    PyTorch caching allocator); otherwise cudaMalloc/cudaFree. All buffers are sized at creation
 *    (capacity, box_capacity); no step allocates.
 */
#ifndef BDM_H
#define BDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BDM_ABI_VERSION 1

typedef enum {
  BDM_OK = 0,
  BDM_EINVAL = -1,   /* invalid argument or parameter                                   */
  BDM_ENOMEM = -2,   /* allocation failed, or capacity / box capacity exceeded           */
  BDM_ECUDA = -3,    /* a CUDA runtime call failed (message names it)                    */
  BDM_ESTATE = -4,   /* a kernel flagged an inconsistent state; the handle is poisoned   */
  BDM_ETIMEOUT = -5, /* a bounded device-side wait ran out                               */
  BDM_EBUDGET = -6   /* request exceeds a memory budget                                  */
} bdm_status;

enum { BDM_MECHANICS = 0, BDM_SIR = 1 };
enum { BDM_FP64 = 0, BDM_MIXED = 1 };

/* Simulation parameters.  Zero-initialise, then set struct_size = sizeof(bdm_params). */
typedef struct bdm_params {
  uint32_t struct_size;          /* = sizeof(bdm_params) (ABI check)                             */
  int32_t kind;                  /* BDM_MECHANICS or BDM_SIR                                      */
  int32_t precision;             /* BDM_FP64: all-FP64 force/update; BDM_MIXED: FP32 forces from
                                    box-relative offsets, FP64 positions                         */
  int32_t record_diagnostics;    /* reserved, 0                                                   */
  /* Mechanics (readings R1-R6: neighbour radius, force law, capped update, grid). */
  double dt;                     /* displacement = dt * summed force                               */
  double repulsion;              /* k in F = k delta - gamma sqrt(rho delta)                       */
  double attraction;             /* gamma                                                          */
  double max_displacement;       /* cap on |displacement| per step                                 */
  double interaction_radius;     /* neighbour radius R; 0 = largest diameter, every step.  With
                                    BDM_MIXED, R must be at least the largest diameter (contacts
                                    are found among the pairs within R); a step that finds a
                                    larger diameter fails with BDM_ESTATE                        */
  double box_length;             /* grid box L >= R + skin; 0 = R + skin                           */
  double skin;                   /* neighbour-list skin (mixed precision without growth; 0 = off):
                                    the grid is rebuilt and each agent's candidates within R + skin
                                    are listed only when some agent has moved more than skin / 2
                                    since the last rebuild (or after 64 steps); the steps between
                                    evaluate the lists.  Integer state stays exact every step; the
                                    FP32 force sums follow the order of the last rebuild.  A tiny
                                    skin (e.g. 0.001 um) rebuilds every step through the list
                                    kernels, faster than skin 0's walk at 1e7-1e8 agents.          */
  /* Growth and division (reading R7). */
  int32_t growth_enabled;
  int32_t force_variant;         /* mixed force kernel: 0 = one thread per agent, 1 = warp-shared
                                    (agent, candidate) pairs; same results (tunable)              */
  double growth_volume;          /* volume added per step                                          */
  double division_volume;        /* divide when volume >= this                                     */
  double division_offset_frac;   /* mother/daughter offset = frac * daughter diameter             */
  /* Substance grid: secretion (R8) and FTCS diffusion (R9). */
  int32_t diffusion_enabled;     /* co-step one FTCS step after mechanics in bdm_step              */
  int32_t grid_n[3];             /* voxels per axis (x, y, z); layout x fastest                    */
  double grid_origin[3];
  double voxel;                  /* h                                                              */
  double diffusion_coeff;        /* D                                                              */
  double decay;                  /* mu                                                             */
  double dt_diffusion;           /* dt of one FTCS step                                            */
  double secretion;              /* amount each agent adds per step; 0 = none                      */
  /* SIR (reading R10); lengths in um, run on a 2^-10 um int32 lattice. */
  double sir_domain;             /* periodic cube side L                                           */
  double sir_radius;             /* infection radius r                                             */
  double sir_step;               /* per-axis move bound s                                          */
  double p_infect;
  double p_recover;
  int32_t sir_boxes;             /* boxes per axis nb (L / nb >= r, nb divides the lattice side);
                                    0 = largest admissible box count <= L / r                    */
  int32_t reserved2;
  /* Random streams: Philox4x32-10 key = (seed low 32 bits, run_id). */
  uint64_t seed;
  uint32_t run_id;
  uint32_t reserved3;
  /* Capacities. */
  uint64_t capacity;             /* max agents (growth appends up to it); 0 = agents of the first
                                    bdm_add_agents call                                           */
  uint64_t box_capacity;         /* max grid boxes; 0 = automatic (4 x initial + margin)           */
  /* Stationary agents (skin > 0): on a list step a warp-sized group of agents (32 consecutive in
     the sorted order) whose agents, and every agent in the boxes around them, kept their positions
     in the previous step would get the same forces, displacements (zero) and neighbour counts
     again, so it is left out.  The results are identical either way. */
  int32_t skip_stationary;       /* 1 = skip such groups; 0 = evaluate every agent every step     */
  int32_t reserved4;
  /* Oncology behaviours (readings R13, R14; the grid is then rebuilt every step, skin = 0). */
  double brownian_sigma;         /* Brownian migration: after the capped mechanical update every
                                    agent moves by sigma * N(0,1) per axis (um); 0 = off          */
  double p_apoptosis;            /* each agent dies at the start of a step with this probability;
                                    survivors keep their order and take dense ids; 0 = off       */
  double chemotaxis;             /* chi (reading R15, needs the substance grid): after the update
                                    every agent moves by chi * grad c at its step-start voxel of
                                    the step-start grid (um per unit of c per um); 0 = off        */
  /* Device plumbing. */
  void* stream;                  /* cudaStream_t, NULL = a stream the handle creates              */
  void* (*alloc)(size_t bytes, void* user); /* optional device allocator                         */
  void (*free)(void* ptr, void* user);
  void* alloc_user;
} bdm_params;

/* Read-out of one simulation.  Set struct_size; every pointer may be NULL (field skipped); buffers
 * must hold at least `n` entries (query n first with all pointers NULL), grid prod(grid_n).  A
 * field that the handle's kind does not hold (diameter and volume for SIR; sir_state for
 * mechanics; volume without growth) is not written: its buffer keeps what the caller put there. */
typedef struct bdm_state {
  uint32_t struct_size;          /* = sizeof(bdm_state)                                            */
  uint32_t reserved0;
  uint64_t n;                    /* out: number of agents                                          */
  uint64_t step;                 /* out: steps completed                                           */
  double* x;                     /* positions, um                                                   */
  double* y;
  double* z;
  float* diameter;               /* mechanics                                                      */
  double* volume;                /* mechanics with growth                                          */
  uint8_t* sir_state;            /* SIR: 0 susceptible, 1 infected, 2 recovered                    */
  uint32_t* neighbour_count;     /* last step: mechanics -> agents within R; SIR -> infected
                                    agents within r (both at step start)                          */
  uint32_t* box_id;              /* last step's grid assignment of each agent                      */
  float* grid;                   /* substance grid, x fastest                                      */
  double mass_total;             /* out: FP64 total of the substance grid                          */
  uint32_t sir_counts[3];        /* out: S, I, R after the last step                               */
  uint32_t grid_rebuilds;        /* out: grid rebuilds so far (mechanics; = steps without skin)    */
  int64_t grid_origin_q[3];      /* out: last grid origin, 2^-20 um lattice units (mechanics)      */
  int64_t grid_box_q;            /* out: box length, lattice units                                 */
  int64_t grid_dims[3];          /* out: boxes per axis                                            */
  uint64_t list_entries;         /* out: listed candidates at the last rebuild (skin > 0)          */
  uint64_t stationary_skipped;   /* out: agent evaluations skipped as stationary, all steps so far */
} bdm_state;

typedef struct bdm_sim bdm_sim;

/* Create a simulation handle.  Validates p (BDM_EINVAL), allocates device state for p->capacity
 * agents (or defers to the first bdm_add_agents when 0) and p->box_capacity boxes. */
int bdm_create(const bdm_params* p, bdm_sim** out);

/* Append n agents (ids continue from the current count).  x, y, z: host arrays of n doubles (um).
 * diameter: n floats (mechanics; NULL for SIR).  volume: n doubles or NULL (then pi/6 d^3).
 * sir_state: n bytes or NULL (all susceptible).  SIR positions must lie in [0, sir_domain) and are
 * rounded to the 2^-10 um lattice.  BDM_ENOMEM beyond capacity. */
int bdm_add_agents(bdm_sim* s, size_t n, const double* x, const double* y, const double* z,
                   const float* diameter, const double* volume, const uint8_t* sir_state);

/* Replace the substance grid with prod(grid_n) host floats (x fastest). */
int bdm_set_grid(bdm_sim* s, const float* values);

/* Set the step counter (Philox counters are keyed by it); used to resume from a saved state. */
int bdm_set_step(bdm_sim* s, uint64_t step);

/* Remove all agents and zero the step counter, keeping every allocation. */
int bdm_reset(bdm_sim* s);

/* Advance n steps (reading R11 order).  Asynchronous; n-step sequences are captured once into a
 * CUDA graph and replayed. */
int bdm_step(bdm_sim* s, int n);

/* Advance the substance grid alone by n FTCS steps (standalone operation). */
int bdm_diffusion_step(bdm_sim* s, int n);

/* Copy the state to caller buffers in agent-id order.  Synchronises the stream. */
int bdm_get_state(bdm_sim* s, bdm_state* st);

void bdm_destroy(bdm_sim* s);
const char* bdm_last_error(const bdm_sim* s);

/* ---- Profiling: per-kernel CUDA-event timing on the simulation's stream ---------------------- */
typedef struct bdm_kernel_time {
  char name[32];
  uint64_t launches;
  double total_ms;
} bdm_kernel_time;

/* enable != 0: record an event pair around every kernel the handle launches (no graph replay while
 * enabled: steps are issued kernel by kernel). */
int bdm_profile(bdm_sim* s, int enable);
/* Fill up to max entries (synchronises); returns the number of distinct kernels in *count. */
int bdm_kernel_times(bdm_sim* s, bdm_kernel_time* out, int max, int* count);
/* Kernels this process has launched through libbdm (graph replays count each node). */
uint64_t bdm_launch_count(void);
/* Library version string. */
const char* bdm_version(void);

/* ---- Batched SIR ensemble ------------------------------------------------------------------------ */
/* Many SIR simulations (Sec. "Epidemiology use case": runs of the random-walk infection model with
 * their own parameters) advanced together: every step is ONE persistent kernel launch covering all
 * runs (a work list of (run, 256-agent tile) pairs; phases separated by a grid barrier whose waits
 * are bounded), and n-step sequences are captured into a CUDA graph.  Each run computes exactly what
 * a single-run handle would: the arithmetic is integer and per run. */
typedef struct bdm_batch bdm_batch;
typedef struct bdm_batch_options {
  uint32_t struct_size;          /* = sizeof(bdm_batch_options)                                    */
  uint32_t history_steps;        /* S/I/R counts kept per run (ring); 0 = 1024                     */
  uint32_t spin_limit;           /* bounded-wait iterations of the grid barrier (~100 ns each);
                                    0 = default (~0.4 s)                                          */
  uint32_t barrier_extra;        /* test hook, 0 in normal use: arrivals the grid barrier waits for
                                    beyond the launched grid, so that its bounded wait runs out and
                                    the batch reports BDM_ETIMEOUT (no GPU fault)                 */
  void* stream;                  /* cudaStream_t, NULL = a stream the batch creates               */
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* alloc_user;
  uint32_t persistent_only;      /* 1 = always the persistent grid kernel; 0 = one CTA per run
                                    (histogram, scan and counts in shared memory) whenever every
                                    run's nb^3 + 1 + agents words fit in a CTA's shared memory.
                                    Both give the same results.                                   */
  uint32_t reserved0;
} bdm_batch_options;

/* per_sim: `count` parameter blocks with kind = BDM_SIR (their seed/run_id key each run's Philox
 * stream; sir_boxes 0 = about one agent per box).  opt may be NULL. */
int bdm_batch_create(const bdm_params* per_sim, int count, const bdm_batch_options* opt,
                     bdm_batch** out);
/* Append agents (host arrays, um; sir_state NULL = susceptible) to run `sim`; only before the first
 * step (the layout is fixed then). */
int bdm_batch_add_agents(bdm_batch* b, int sim, size_t n, const double* x, const double* y,
                         const double* z, const uint8_t* sir_state);
/* Advance every run by n steps (asynchronous).  A step is one launch per step: one CTA per run
 * when the runs fit in shared memory (see persistent_only), else one persistent grid over all runs. */
int bdm_batch_step(bdm_batch* b, int n);
/* Wait for the batch's stream; BDM_ETIMEOUT if a grid-barrier wait ran out. */
int bdm_batch_sync(bdm_batch* b);
/* One run's state (agent-id order; box_id is run-local), like bdm_get_state. Synchronises. */
int bdm_batch_get_state(bdm_batch* b, int sim, bdm_state* st);
/* S/I/R counts after each of the last min(max_steps, history) steps, oldest first:
 * out[step][run][3]; *steps receives the number of steps written.  Synchronises. */
int bdm_batch_counts(bdm_batch* b, uint32_t* out, int max_steps, int* steps);
void bdm_batch_destroy(bdm_batch* b);
const char* bdm_batch_last_error(const bdm_batch* b);

/* ---- Batched mechanics (served simulations) --------------------------------------------------- */
/* A pool of simulation slots for the plain sphere mechanics (Sec. "Simulation concepts": every step
 * the uniform-grid rebuild, the 27-box neighbour search, the force and the capped update; readings
 * R1-R6).  A slot holds one simulation of up to slot_capacity agents with its own parameters and
 * step target; simulations are loaded into free slots and released between steps at any time
 * (continuous admission).  Every step advances all active slots together in nine launches,
 * whatever the number of simulations: each kernel covers a work list of (slot, 256-agent tile)
 * pairs, and each slot keeps its own grid, agent range and box range.  Steps are captured into a
 * CUDA graph per step count.  Each slot computes what a single handle (bdm_create) computes for the
 * same simulation, which rebuilds the grid every step, bit for bit on both paths (the mixed path's
 * per-pair FP32 operations are explicitly rounded, so no kernel contracts them differently).
 *   precision             BDM_FP64 or BDM_MIXED (every slot)
 *   slots, slot_capacity  pool shape, slots x slot_capacity < 2^31 agents; allocated here: about
 *                         100 B per agent place and 8 B per box place, 2 slot_capacity + 4096 box
 *                         places per slot
 *   stream                cudaStream_t, NULL = a stream the pool creates */
typedef struct bdm_mbatch bdm_mbatch;
int bdm_mbatch_create(int precision, int slots, size_t slot_capacity, void* stream,
                      bdm_mbatch** out);
/* Load a simulation into free slot `slot`: its parameters p (kind BDM_MECHANICS, the pool's
 * precision, no skin, growth, diffusion or oncology behaviours), its n agents (HOST arrays, um;
 * 1 <= n <= slot_capacity; ids 0 .. n - 1 in this order) and the number of steps it runs.  Waits for
 * the pool's stream.  BDM_ESTATE if the slot is occupied; BDM_EINVAL for bad parameters or agents
 * (a diameter <= 0 or |position| >= 1e9 um). */
int bdm_mbatch_load(bdm_mbatch* b, int slot, const bdm_params* p, size_t n, const double* x,
                    const double* y, const double* z, const float* diameter, int steps);
/* Advance every active slot by n steps (a slot stops at its step target); asynchronous. */
int bdm_mbatch_step(bdm_mbatch* b, int n);
/* Steps completed by each slot into steps_done[slots] (-1 for a free slot).  Waits for the stream. */
int bdm_mbatch_poll(bdm_mbatch* b, int32_t* steps_done);
/* One slot's state in agent-id order (box ids on the slot's grid of its last step), like
 * bdm_get_state; grid_rebuilds = the slot's steps.  Waits for the stream.  BDM_ENOMEM if the slot's
 * grid needed more boxes than it holds, BDM_ESTATE for another grid failure. */
int bdm_mbatch_get_state(bdm_mbatch* b, int slot, bdm_state* st);
/* Free a slot for the next simulation (its state is discarded).  Waits for the stream. */
int bdm_mbatch_release(bdm_mbatch* b, int slot);
void bdm_mbatch_destroy(bdm_mbatch* b);
const char* bdm_mbatch_last_error(const bdm_mbatch* b);

/* ---- Utility ----------------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11), the counter-based generator behind division axes and the SIR
 * behaviours, evaluated by the library's device code.  ctr: n x 4 words, key: n x 2 words, out:
 * n x 4 words, all HOST arrays (row-major).  Allocates temporary device memory.  Used to check the
 * device generator against independent implementations. */
int bdm_philox(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* ---- Allocation-free diffusion step -------------------------------------------------------- */
/* One FTCS step (same arithmetic as the diffusion co-step of bdm_step) for callers that cannot
 * allocate device memory: applications that hand all device memory out of their own pool, code
 * running while another framework captures a CUDA graph, or loops that cannot afford the implicit
 * synchronisation of cudaMalloc/cudaFree.  The paper has no counterpart; this is an interface
 * variant of the library.
 *   u, out   DEVICE grids of prod(grid_n) floats (x fastest), caller-owned, distinct.
 *   grid_n   voxels per axis (host array); diffusion_coeff, dt_diffusion, voxel, decay as in
 *            bdm_params (the step must be stable: D dt / h^2 <= 1/6).
 *   mass     DEVICE double that receives the FP64 total of `out`, or NULL.
 *   stream   cudaStream_t (NULL = legacy default stream); the call is asynchronous.
 * Allocates nothing: its scratch is a static device array of 65,536 doubles (512 KB per GPU that
 * loads the library), so grids needing more than 65,536 blocks of 32 x 8 x 16 voxels are rejected
 * with BDM_EINVAL (e.g. 512^3 uses 32,768), as are grids beyond the launch limits (more than
 * 65,535 blocks along y or z).  The first call on a device looks up that array's address once, in
 * the device's primary context, and keeps it for the life of the process: make that call before any
 * stream capture, and do not use the entry point after cudaDeviceReset or from a context other than
 * the primary one (the array lives at another address there).  All calls share the array: calls that overlap
 * on the GPU race on it, so order them (one stream, or events).  Returns BDM_EINVAL for bad
 * arguments, BDM_ECUDA if the launch fails. */
int bdm_diffusion_step_noalloc(const float* u, float* out, const int32_t grid_n[3],
                               double diffusion_coeff, double dt_diffusion, double voxel,
                               double decay, double* mass, void* stream);

#ifdef __cplusplus
}
#endif
#endif
