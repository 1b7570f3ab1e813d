/*
 * oracle.h -- plain FP64 CPU oracle for the agent-mechanics step (TEST INFRASTRUCTURE).
 *
 * This library is the independent reference that the CUDA path is checked against. It is slow on
 * purpose: every function is a direct loop over the definition. Only tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product library never links or calls it, and it
 * shares no source with the product library.
 *
 * Model sources (BioDynaMo, arXiv 2006.06775):
 *   - uniform grid, 27-box environment, box size from the largest agent: Section "Simulation
 *     concepts" (environment paragraph) and Fig. 1C;
 *   - agent operations (behaviours, mechanical forces) vs standalone operations (diffusion):
 *     Section "Simulation concepts" (operations paragraph);
 *   - sphere-sphere force: the paper states only that it uses the Cortex3D method (Section
 *     "Performance"); the law used here (readings R1-R4) is stated beside orc_mech_step;
 *   - SIR behaviours and counting operation: Section "Epidemiology use case";
 *   - neurite elements (cylinders with a spring and a distal point mass, joined as trees): Section
 *     "Neuroscience module"; their contact law (readings R16-R20) is stated beside
 *     orc_neurite_step in oracle.c.
 *
 * Conventions: all arrays are caller-owned, in agent-id order unless stated; functions return 0 on
 * success and a negative code on invalid input (-1) or allocation failure (-2).
 */
#ifndef BDM_ORACLE_H
#define BDM_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): one block of four 32-bit words. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* n independent blocks: ctr is n x 4, key is n x 2, out is n x 4 (row-major). */
void orc_philox4x32_10_n(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* Uniform grid of one step (reading R5).  Output vector g (10 doubles):
 * g[0..2] origin, g[3] interaction radius, g[4] box length, g[5] 1/box length,
 * g[6..8] boxes per axis, g[9] number of boxes. */
int orc_grid(size_t n, const double* x, const double* y, const double* z, const float* diam,
             double interaction_radius, double box_length, double* g, uint32_t* box_id);

typedef struct {
  double dt;                 /* time step of the displacement update                          */
  double k_rep;              /* repulsion coefficient k                                       */
  double gamma_att;          /* attraction coefficient gamma                                  */
  double max_disp;           /* displacement cap (norm)                                       */
  double interaction_radius; /* neighbour radius; 0 = largest diameter                        */
  double box_length;         /* grid box; 0 = interaction radius; must be >= it otherwise     */
} orc_mech_params;

/* One Jacobi step of sphere mechanics: grid rebuild, 27-box neighbour search, force sum in the
 * canonical (box, id) order, capped displacement update.  Writes new positions, the neighbour count
 * of each agent (agents j != i with |x_i - x_j|^2 < R^2), the box id of each agent and the grid
 * vector g (see orc_grid).  fx/fy/fz (may be NULL) receive the summed force of each agent. */
int orc_mech_step(size_t n, const double* x, const double* y, const double* z, const float* diam,
                  const orc_mech_params* p, double* nx, double* ny, double* nz, uint32_t* nbr,
                  uint32_t* box_id, double* g, double* fx, double* fy, double* fz);

/* Growth and division behaviour (reading R7).  Agents 0..n-1 grow by dv; those with volume >= vdiv
 * divide.  Arrays have room for 2n agents; daughters are appended at ids n + rank.  Returns the new
 * agent count through n_out.  Key = (seed_lo, run), counter = (id, step, 2, attempt). */
int orc_grow_divide(size_t n, double* x, double* y, double* z, float* diam, double* vol,
                    double dv, double vdiv, double offset_frac, uint32_t seed_lo, uint32_t run,
                    uint32_t step, size_t* n_out);
/* Apoptosis at step start (reading R14): removes the agents that die, keeps the order; returns m. */
size_t orc_apoptosis(size_t n, double* x, double* y, double* z, float* diam, double* vol,
                     uint64_t thr, uint32_t seed_lo, uint32_t run, uint32_t step);
/* Brownian migration after the mechanical update (reading R13). */
void orc_brownian(size_t n, double* x, double* y, double* z, double sigma, uint32_t seed_lo,
                  uint32_t run, uint32_t step);
/* Chemotaxis after the update (reading R15): x += chi * grad c at the step-start voxel. */
void orc_chemotaxis(size_t n, double* x, double* y, double* z, const double* sx, const double* sy,
                    const double* sz, const double* grid, const int64_t dims[3],
                    const double origin[3], double h, double chi);

/* Secretion (reading R8): each agent adds q to the voxel that holds its centre (clamped). */
void orc_secrete(size_t n, const double* x, const double* y, const double* z, double* grid,
                 const int64_t dims[3], const double origin[3], double h, double q);

/* One explicit 7-point FTCS step with zero-flux walls and linear decay (reading R9):
 * out = u + lambda * sum_nb (u_nb - u) - mu_dt * u.  Returns the FP64 mass of out. */
double orc_ftcs(const int64_t dims[3], const double* u, double* out, double lambda, double mu_dt);

/* One synchronous SIR step of one run (reading R10).  Positions are int32 fixed point in a periodic
 * cube of side L (same units), nb boxes per axis (L % nb == 0, L / nb >= r).  state: 0 S, 1 I, 2 R.
 * Writes new positions/state, the number of infected agents within r of each agent (at step
 * start), each agent's box id, and the S/I/R counts after the step. */
int orc_sir_step(size_t n, const int32_t* X, const int32_t* Y, const int32_t* Z, const uint8_t* st,
                 int32_t L, int32_t nb, int32_t r, int32_t s, uint64_t thr_inf, uint64_t thr_rec,
                 uint32_t seed_lo, uint32_t run, uint32_t step, int32_t* nX, int32_t* nY,
                 int32_t* nZ, uint8_t* nst, uint32_t* ninf, uint32_t* box_id, uint32_t counts[3]);

/* Neurite mechanics (readings R16-R20): somata (mother < 0, spheres) and neurite elements
 * (cylinders from p_mother + o to p).  mother[a] < a for every element (a tree in creation order).
 * Brute force over all pairs.  Writes new positions, neighbour counts (R20), the radius L used
 * (L_out, may be NULL) and, when fx is not NULL, each agent's total force. */
typedef struct {
  double dt, k_rep, gamma_att, max_disp;
  double k_spring;            /* spring constant of an element (R17)                  */
  double interaction_radius;  /* lower bound of L; 0 = the largest extent (R20)       */
} orc_neurite_params;

void orc_segment_closest(const double P0[3], const double u[3], const double Q0[3],
                         const double v[3], double* s_out, double* t_out);
int orc_neurite_step(size_t n, const double* x, const double* y, const double* z,
                     const double* diam, const double* rest, const int32_t* mother,
                     const double* ox, const double* oy, const double* oz,
                     const orc_neurite_params* p, double* nx, double* ny, double* nz,
                     uint32_t* nbr, double* L_out, double* fx, double* fy, double* fz);
/* The same step for the m agents idx[0..m-1] only (new positions and counts in sample order). */
int orc_neurite_sample(size_t n, const double* x, const double* y, const double* z,
                       const double* diam, const double* rest, const int32_t* mother,
                       const double* ox, const double* oy, const double* oz,
                       const orc_neurite_params* p, size_t m, const int64_t* idx, double* nx,
                       double* ny, double* nz, uint32_t* nbr, double* L_out);

/* Threads the OpenMP build uses (1 without OpenMP). */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
