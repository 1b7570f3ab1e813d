/*
 * bdm_neurite.h -- C ABI of the neurite-mechanics path in libbdm.so (sm_103a).
 *
 * BioDynaMo (arXiv 2006.06775), Sec. "Neuroscience module": a neuron is a soma (a sphere) with
 * neurites made of neurite elements; an element is a cylinder, modelled as a spring with a point
 * mass at its distal end, and elements form a binary tree through which forces are passed along
 * the chain.  Sec. "Simulation concepts" gives agents sphere or cylinder geometry and a uniform grid
 * whose box length is set by the largest agent.  The paper prints no cylinder force law; this path
 * computes the following readings (the FP64 oracle states the same):
 *   R16 agent a is a soma (mother[a] < 0: a sphere centred at p_a) or an element: a cylinder from
 *       the proximal point q_a = p_{mother[a]} + o_a to the distal point p_a, radius d_a / 2;
 *   R17 spring: v = p_e - q_e, l = |v|, T = spring * (l - rest_e) / rest_e; the element's distal
 *       point takes -T v / l and its mother +T v / l;
 *   R18 contact: the closest points of the two bodies (the argmin of the distance between the
 *       two axes; parallel axes, whose minimum is not unique, take the first of the edge
 *       minimisers s = 0, s = 1, t = 0, t = 1 that attains it), then the sphere law F = k delta -
 *       gamma sqrt(rho delta) (delta = r_i + r_j - distance, rho = r_i r_j / (r_i + r_j)) along the
 *       line between them when delta > 0; an element at axial parameter s (0 proximal, 1 distal)
 *       keeps s of the force at its distal point and passes 1 - s to its mother;
 *   R19 no contact between an element and its mother or daughters, or between two elements with
 *       the same mother (they share an end point);
 *   R20 neighbours of i: agents j != i whose binning points (soma: centre; element: midpoint) are
 *       closer than L, L = the largest extent (soma: diameter; element: length + diameter) or
 *       interaction_radius if larger; grid boxes are L (widened by 2^-20) wide, so the 27 boxes
 *       around an agent hold every neighbour and every contact;
 *   update (R4): D = dt * (own share + the shares passed up by its daughters, in ascending daughter
 *       id), scaled to max_displacement if longer, p += D; all agents from the step-start state.
 *
 * Conventions as in bdm.h: 0 / negative bdm_status, host pointers copied before the call returns,
 * work enqueued on the handle's stream (bdm_neurite_get_state synchronises it), device error bits
 * surfacing at the next synchronising call.  Agents keep their ids (insertion order) across steps.
 */
#ifndef BDM_NEURITE_H
#define BDM_NEURITE_H

#include <stddef.h>
#include <stdint.h>

#include "bdm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bdm_neurite_params {
  uint32_t struct_size;        /* = sizeof(bdm_neurite_params)                                  */
  int32_t precision;           /* BDM_FP64: contacts in FP64 (the check path); BDM_MIXED: contact
                                  geometry in FP32 from box-relative offsets, FP64 positions,
                                  springs and neighbour decisions                               */
  double dt;                   /* displacement = dt * summed force                               */
  double repulsion;            /* k                                                              */
  double attraction;           /* gamma                                                          */
  double max_displacement;     /* cap on |displacement| per step                                 */
  double spring;               /* spring constant of an element (R17)                            */
  double interaction_radius;   /* lower bound of L (R20); 0 = the largest extent                 */
  uint64_t capacity;           /* agents the handle can hold (at most 2^31; 2^27 with BDM_MIXED) */
  uint64_t box_capacity;       /* grid boxes; 0 = 2 * capacity + 4096.  A step whose grid needs
                                  more fails with BDM_ENOMEM at the next synchronising call       */
  void* stream;                /* cudaStream_t, NULL = a stream the handle creates               */
  double skin;                 /* >= 0.  BDM_MIXED only: 0 = the grid is rebuilt every step (the
                                  paper's cadence); > 0 = neighbour lists.  A rebuild step bins
                                  the agents on boxes of L + skin and lists, per agent, every
                                  other agent whose binning point lies within L + skin; the steps
                                  after it evaluate the lists (same counts, contacts and update)
                                  until a binning point may have moved more than
                                  (skin - (L - L_rebuild)) / 2 since the rebuild (the summed
                                  displacement of the agent's own point bounds that of its
                                  binning point), after 64 steps, or after set_agents.  The FP32
                                  contact sums then follow the list order of the last rebuild.  */
} bdm_neurite_params;

typedef struct bdm_neurite bdm_neurite;

/* Validate p (BDM_EINVAL) and allocate the device state (BDM_ENOMEM / BDM_ECUDA). */
int bdm_neurite_create(const bdm_neurite_params* p, bdm_neurite** out);

/* Replace the agents with n new ones (ids 0..n-1).  x/y/z: soma centre or element distal point;
 * diameter > 0; rest > 0 for elements (ignored for somata); mother: -1 for a soma, else the
 * mother's id, smaller than the agent's own (a tree in creation order); ox/oy/oz: the offset of the
 * proximal point from the mother's point (ignored for somata).  BDM_EINVAL for a rejected agent
 * (the message names it), BDM_ENOMEM beyond capacity. */
int bdm_neurite_set_agents(bdm_neurite* s, size_t n, const double* x, const double* y,
                           const double* z, const double* diameter, const double* rest,
                           const int32_t* mother, const double* ox, const double* oy,
                           const double* oz);

/* Enqueue n steps (asynchronous; n >= 0). */
int bdm_neurite_step(bdm_neurite* s, int n);

/* Synchronise and copy the state in id order.  Every pointer may be NULL.  n_out: agents; x/y/z:
 * positions (n each); neighbour_count: R20 counts of the last step (n); L_out: its radius L.
 * Before the first step after bdm_neurite_set_agents the counts and L read 0. */
int bdm_neurite_get_state(bdm_neurite* s, size_t* n_out, double* x, double* y, double* z,
                          uint32_t* neighbour_count, double* L_out);

/* Neighbour-list bookkeeping (skin > 0; synchronises the stream): rebuilds since the last
 * bdm_neurite_set_agents (or NULL) and the entries listed by the last rebuild (or NULL).  Both
 * read 0 without a skin. */
int bdm_neurite_list_info(bdm_neurite* s, uint64_t* rebuilds, uint64_t* entries);

/* Per-kernel CUDA-event timing of later steps (as bdm_profile / bdm_kernel_times). */
int bdm_neurite_profile(bdm_neurite* s, int enable);
int bdm_neurite_kernel_times(bdm_neurite* s, bdm_kernel_time* out, int max, int* count);

void bdm_neurite_destroy(bdm_neurite* s);
const char* bdm_neurite_last_error(const bdm_neurite* s);

#ifdef __cplusplus
}
#endif
#endif
