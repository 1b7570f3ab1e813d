// sir.cuh -- device-side layout of the SIR model (single run and batched ensemble).
#pragma once
#include "common.cuh"

namespace bdm {

// Per-run constants (reading R10), in 2^-10 um lattice units.
struct SirRun {
  int L;                        // periodic cube side
  int nb;                       // boxes per axis
  int Lb;                       // box side = L / nb (>= r)
  float invLb;                  // float(1 / Lb): estimate for the box division
  int s;                        // move bound per axis
  unsigned long long span;      // 2 s + 1
  long long r2;                 // infection radius squared
  unsigned long long thr_inf;   // floor(p_inf * 2^32)
  unsigned long long thr_rec;   // floor(p_rec * 2^32)
  uint2 key;                    // Philox key (seed low word, run id)
  unsigned agent_off, agent_n;  // agents of this run: [agent_off, agent_off + agent_n)
  unsigned box_off;             // boxes of this run: [box_off, box_off + nb^3)
};

// The agents, in id order, updated in place.
struct SirState {
  int *X, *Y, *Z;
  unsigned char* st;
};

// Per-agent and per-box buffers (one run, or a batch of concatenated runs):
//   kn/rk   box of each agent at the start of the coming step (global box index) and its rank in
//           that box; the update writes them together with the box histogram `count`
//   perm    agents in box order (start[box] .. start[box + 1])
//   src     this step's infected agents as (agent, run)
//   ninf    infected agents within the radius of each agent (read-out and infection input)
//   box     read-out: box of each agent at the start of the last step
struct SirSingle {
  SirState a;
  unsigned *kn, *rk, *perm, *count, *start, *ninf, *box;
  uint2* src;
  unsigned long long* tiles;
  unsigned max_tiles;
  SirRun run;
};

struct SirBatchDev {
  SirState a;
  unsigned *kn, *rk, *perm, *count, *start, *ninf, *box;
  uint2* src;
  unsigned long long* tiles;
  unsigned max_tiles;
  const SirRun* run;            // [runs]
  const unsigned* tile_run;     // work list: run of each 256-agent tile
  const unsigned* tile_start;   // work list: first agent of each tile
  unsigned ntiles, runs, total_agents, total_boxes;
  unsigned* hist;               // [hist_len][runs][3] S/I/R after each step
  unsigned hist_len;
  unsigned* bar;                // grid barrier: [0] arrivals, [1] generation
};

// Boxes per axis of a SIR grid: the given count, else the largest divisor of the lattice side L
// (lattice units) that keeps the box side >= r and puts about one agent in a box.
inline int sir_box_count(long long L, long long r, int given, size_t n) {
  if (given > 0) return given;
  long long limit = r > 0 ? L / r : L;
  long long target = 1;
  while ((target + 1) * (target + 1) * (target + 1) <= (long long)(n > 0 ? n : 1)) ++target;
  if (target < limit) limit = target;
  for (long long nb = limit > 1 ? limit : 1; nb >= 1; --nb)
    if (L % nb == 0) return (int)nb;
  return 1;
}

// Box, rank and histogram entry of agents [lo, hi) of a single run before their first step.
void launch_sir_init(cudaStream_t s, const SirSingle& S, unsigned lo, unsigned hi, int grid_blocks);
// Same for every agent of a batch.
void launch_sir_init_batch(cudaStream_t s, const SirBatchDev& B, int grid_blocks);
void launch_sir_step(cudaStream_t s, const SirSingle& S, DevGrid* g, int grid_blocks, int scan_blocks);
cudaError_t launch_sir_ensemble(cudaStream_t s, const SirBatchDev& B, DevGrid* g, int blocks,
                                unsigned barrier_extra, unsigned spin_limit, bool cooperative);
int sir_ensemble_blocks_per_sm();
// One CTA per run (histogram, scan and counts in shared memory); sir_runs_smem_bytes returns the
// dynamic shared memory for runs of up to `words` = nb^3 + 1 + agents words, or 0 if it does not fit.
size_t sir_runs_smem_bytes(size_t words);
void launch_sir_runs(cudaStream_t s, const SirBatchDev& B, DevGrid* g, size_t smem_bytes);
void launch_philox(cudaStream_t s, unsigned n, const uint4* ctr, const uint2* key, uint4* out);

}  // namespace bdm
