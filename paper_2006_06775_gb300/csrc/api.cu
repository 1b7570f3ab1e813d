// api.cu -- the C ABI of libbdm (declared and documented in include/bdm.h).
//
// A handle owns the device state of one simulation (BioDynaMo, arXiv 2006.06775, Sec. "Simulation
// concepts": define the model -- agents, attributes, behaviours -- then execute operations step by
// step).  Every step is enqueued on the handle's stream without host round trips (the grid
// description lives in device memory), so an n-step sequence is captured once into a CUDA graph and
// replayed.  Device-side error bits are polled asynchronously and surface at the next call.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "bdm.h"
#include "common.cuh"
#include "sir.cuh"

using namespace bdm;

static std::atomic<unsigned long long> g_launches{0};

// Kernel launches issued by other parts of the library (batched ensembles).
void bdm_count_launches(unsigned long long k) { g_launches += k; }

namespace {

struct KernelStat {
  std::string name;
  uint64_t launches = 0;
  double total_ms = 0.0;
};

struct Profiler {
  bool on = false;
  struct Pending {
    int stat;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  std::vector<KernelStat> stats;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  int index(const char* name) {
    for (size_t i = 0; i < stats.size(); ++i)
      if (stats[i].name == name) return (int)i;
    stats.push_back(KernelStat{name, 0, 0.0});
    return (int)stats.size() - 1;
  }
  void resolve() {
    for (auto& p : pending) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, p.a, p.b);
      stats[p.stat].launches += 1;
      stats[p.stat].total_ms += ms;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  ~Profiler() {
    for (auto& p : pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;
  int attr_cur = 0, grid_cur = 0, pos_cur = 0;
  bool bounds_fresh = false;
};

}  // namespace

struct bdm_sim {
  bdm_params p{};
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t copy_stream = nullptr;          // read-out: host copies beside the permutation
  cudaEvent_t axis_done[3] = {nullptr, nullptr, nullptr};
  bool poisoned = false;
  bool allocated = false;
  int sms = 152;
  size_t capacity = 0, box_capacity = 0;
  size_t n_host = 0;       // agents as known to the host (growth: refreshed at sync points)
  bool growth = false, mixed = false, is_sir = false, diffusion = false;
  DevGrid* g = nullptr;
  DevGrid* gh = nullptr;    // pinned host mirror
  unsigned* err_pinned = nullptr;
  cudaEvent_t err_event = nullptr;
  bool err_pending = false;
  MechBuffers mb{};
  MechConsts mc{};
  int attr_cur = 0;
  int pos_cur = 0;          // skin > 0: the position set holding the current agents
  bool bounds_fresh = false;
  float* grid[2] = {nullptr, nullptr};
  int grid_cur = 0;
  double* partials = nullptr;
  int gdims[3] = {0, 0, 0};
  float lam = 0.f, mu_dt = 0.f;
  SirSingle sb{};
  std::vector<void*> allocs;
  // n-step graphs keyed by (steps, diffusion only, attr parity, grid parity, bounds fresh, SIR
  // agent count, position-set parity): each key fixes every pointer and launch size the capture saw
  std::map<std::tuple<int, int, int, int, int, size_t, int>, GraphEntry> graphs;
  Profiler prof;
  bool capturing = false;
  unsigned long long capture_kernels = 0;
  int blocks_stream = 1216, blocks_force = 608, blocks_walk = 608, blocks_list = 912, blocks_scan = 608;
  unsigned n_stage = 0;     // host source of the agent-count upload
};

namespace {

int fail(bdm_sim* s, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(s, BDM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int dalloc(bdm_sim* s, void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* q = nullptr;
  if (s->p.alloc) {
    q = s->p.alloc(bytes, s->p.alloc_user);
  } else if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    q = nullptr;
  }
  if (!q) return fail(s, BDM_ENOMEM, "device allocation of %zu bytes failed", bytes);
  s->allocs.push_back(q);
  *ptr = q;
  return BDM_OK;
}

template <typename T>
int dalloc_n(bdm_sim* s, T** ptr, size_t count) {
  return dalloc(s, (void**)ptr, count * sizeof(T));
}

// Launch accounting + optional per-kernel event timing around one launch wrapper call.
template <typename F>
int run(bdm_sim* s, const char* name, unsigned kernels, F&& f) {
  cudaEvent_t a = nullptr, b = nullptr;
  int stat = -1;
  if (s->prof.on && !s->capturing) {
    stat = s->prof.index(name);
    a = s->prof.get();
    b = s->prof.get();
    cudaEventRecord(a, s->stream);
  }
  f();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(s, BDM_ECUDA, "launch of %s failed: %s", name, cudaGetErrorString(e));
  if (s->capturing) s->capture_kernels += kernels;
  else g_launches += kernels;
  if (stat >= 0) {
    cudaEventRecord(b, s->stream);
    s->prof.pending.push_back(Profiler::Pending{stat, a, b});
  }
  return BDM_OK;
}

#define RUN(name, k, body)                                  \
  do {                                                      \
    int rc_ = run(s, name, k, [&]() { body; });             \
    if (rc_) return rc_;                                    \
  } while (0)

unsigned scan_tiles_for(size_t items) { return (unsigned)((items + kScanTile - 1) / kScanTile) + 1u; }

// ---- parameter checks -------------------------------------------------------------------------
int check_params(bdm_sim* s, const bdm_params* p) {
  if (!p) return fail(s, BDM_EINVAL, "params is NULL");
  if (p->struct_size != sizeof(bdm_params))
    return fail(s, BDM_EINVAL, "params.struct_size %u != sizeof(bdm_params) %zu", p->struct_size,
                sizeof(bdm_params));
  if (p->kind != BDM_MECHANICS && p->kind != BDM_SIR) return fail(s, BDM_EINVAL, "unknown kind");
  if (p->kind == BDM_MECHANICS) {
    if (p->precision != BDM_FP64 && p->precision != BDM_MIXED)
      return fail(s, BDM_EINVAL, "unknown precision");
    if (!(p->dt >= 0.0) || !std::isfinite(p->dt)) return fail(s, BDM_EINVAL, "dt must be >= 0");
    if (!(p->max_displacement > 0.0)) return fail(s, BDM_EINVAL, "max_displacement must be > 0");
    if (!(p->repulsion >= 0.0) || !(p->attraction >= 0.0) || !std::isfinite(p->repulsion) ||
        !std::isfinite(p->attraction))
      return fail(s, BDM_EINVAL, "repulsion/attraction must be finite and >= 0");
    if (!(p->interaction_radius >= 0.0) || !(p->box_length >= 0.0))
      return fail(s, BDM_EINVAL, "interaction_radius/box_length must be >= 0");
    if (p->force_variant != 0 && p->force_variant != 1)
      return fail(s, BDM_EINVAL, "force_variant must be 0 or 1");
    if (!(p->skin >= 0.0) || !std::isfinite(p->skin)) return fail(s, BDM_EINVAL, "skin must be >= 0");
    if (p->box_length > 0.0 && p->interaction_radius > 0.0 &&
        p->box_length < p->interaction_radius + p->skin)
      return fail(s, BDM_EINVAL, "box_length below interaction_radius + skin");
    if (!(p->brownian_sigma >= 0.0) || !std::isfinite(p->brownian_sigma))
      return fail(s, BDM_EINVAL, "brownian_sigma must be finite and >= 0");
    if (!(p->p_apoptosis >= 0.0 && p->p_apoptosis <= 1.0))
      return fail(s, BDM_EINVAL, "p_apoptosis must be in [0, 1]");
    if (!std::isfinite(p->chemotaxis)) return fail(s, BDM_EINVAL, "chemotaxis must be finite");
    if (p->chemotaxis != 0.0 && !p->diffusion_enabled)
      return fail(s, BDM_EINVAL, "chemotaxis needs the substance grid (diffusion_enabled)");
    if (p->skin > 0.0 && (p->precision != BDM_MIXED || p->growth_enabled || p->force_variant != 0 ||
                          p->brownian_sigma > 0.0 || p->p_apoptosis > 0.0 || p->chemotaxis != 0.0))
      return fail(s, BDM_EINVAL, "a neighbour-list skin needs mixed precision, force_variant 0 and no "
                                 "growth, apoptosis, Brownian migration or chemotaxis");
    if (p->growth_enabled) {
      if (!(p->growth_volume >= 0.0) || !(p->division_volume > 0.0) ||
          !(p->division_offset_frac >= 0.0))
        return fail(s, BDM_EINVAL, "invalid growth/division parameters");
      if (p->capacity == 0) return fail(s, BDM_EINVAL, "growth needs an explicit capacity");
    }
  } else {
    const double Lu = std::nearbyint(p->sir_domain * 1024.0);
    if (!(Lu >= 1.0) || Lu >= 2147483647.0) return fail(s, BDM_EINVAL, "sir_domain out of range");
    if (!(p->sir_radius >= 0.0) || !(p->sir_step >= 0.0) ||
        std::nearbyint(p->sir_step * 1024.0) >= Lu)
      return fail(s, BDM_EINVAL, "sir_radius/sir_step out of range");
    if (!(p->p_infect >= 0.0 && p->p_infect <= 1.0) || !(p->p_recover >= 0.0 && p->p_recover <= 1.0))
      return fail(s, BDM_EINVAL, "probabilities must lie in [0, 1]");
    if (p->sir_boxes < 0) return fail(s, BDM_EINVAL, "sir_boxes must be >= 0");
  }
  if (p->diffusion_enabled) {
    for (int a = 0; a < 3; ++a)
      if (p->grid_n[a] <= 0) return fail(s, BDM_EINVAL, "grid_n must be positive");
    if (!(p->voxel > 0.0) || !(p->diffusion_coeff >= 0.0) || !(p->dt_diffusion >= 0.0) ||
        !(p->decay >= 0.0))
      return fail(s, BDM_EINVAL, "invalid diffusion parameters");
    const double lam = (p->diffusion_coeff * p->dt_diffusion) / (p->voxel * p->voxel);
    if (lam > 1.0 / 6.0) return fail(s, BDM_EINVAL, "FTCS unstable: D dt / h^2 = %g > 1/6", lam);
    if (p->decay * p->dt_diffusion > 1.0) return fail(s, BDM_EINVAL, "decay * dt > 1");
    if (!ftcs_launchable(p->grid_n))
      return fail(s, BDM_EINVAL, "grid_n %d x %d x %d exceeds the FTCS launch limits", p->grid_n[0],
                  p->grid_n[1], p->grid_n[2]);
  }
  return BDM_OK;
}

unsigned long long threshold(double p) {
  return (unsigned long long)std::floor(p * 4294967296.0);
}

// ---- allocation of the device state (first bdm_add_agents, or first step) --------------------
int allocate(bdm_sim* s, size_t n_first, const double* x, const double* y, const double* z,
             const float* d) {
  const bdm_params& p = s->p;
  s->capacity = p.capacity > 0 ? (size_t)p.capacity : std::max<size_t>(n_first, 1);
  if (n_first > s->capacity)
    return fail(s, BDM_ENOMEM, "%zu agents exceed capacity %zu", n_first, s->capacity);
  if (s->capacity > 0xFFFFFFF0ull) return fail(s, BDM_EINVAL, "capacity above 2^32 agents");
  const size_t C = s->capacity;
  CK(cudaMallocHost((void**)&s->gh, sizeof(DevGrid)));
  CK(cudaMallocHost((void**)&s->err_pinned, sizeof(unsigned)));
  CK(cudaEventCreateWithFlags(&s->err_event, cudaEventDisableTiming));
  int rc = dalloc_n(s, &s->g, 1);
  if (rc) return rc;
  std::memset(s->gh, 0, sizeof(DevGrid));
  for (int a = 0; a < 3; ++a) {
    s->gh->acc_min[a] = ~0ull;
    s->gh->acc_max[a] = 0ull;
  }
  s->gh->nbox1 = 1;
  if (s->is_sir) {
    const int nb = sir_box_count(std::llrint(p.sir_domain * 1024.0), std::llrint(p.sir_radius * 1024.0),
                                 p.sir_boxes, n_first);
    const long long Lu = std::llrint(p.sir_domain * 1024.0);
    const long long ru = std::llrint(p.sir_radius * 1024.0);
    if (Lu % nb != 0 || Lu / nb < ru)
      return fail(s, BDM_EINVAL, "sir_boxes %d must divide the lattice side and keep box >= r", nb);
    SirRun& r = s->sb.run;
    r.L = (int)Lu;
    r.nb = nb;
    r.Lb = (int)(Lu / nb);
    r.invLb = 1.0f / (float)r.Lb;
    r.s = (int)std::llrint(p.sir_step * 1024.0);
    r.span = 2ull * (unsigned long long)r.s + 1ull;
    r.r2 = ru * ru;
    r.thr_inf = threshold(p.p_infect);
    r.thr_rec = threshold(p.p_recover);
    r.key = make_uint2((unsigned)(p.seed & 0xFFFFFFFFull), p.run_id);
    r.agent_off = 0;
    r.agent_n = 0;
    r.box_off = 0;
    const size_t nbox = (size_t)nb * nb * nb;
    s->box_capacity = nbox;
    SirSingle& S = s->sb;
    if ((rc = dalloc_n(s, &S.a.X, C)) || (rc = dalloc_n(s, &S.a.Y, C)) || (rc = dalloc_n(s, &S.a.Z, C)) ||
        (rc = dalloc_n(s, &S.a.st, C)) || (rc = dalloc_n(s, &S.kn, C)) || (rc = dalloc_n(s, &S.rk, C)) ||
        (rc = dalloc_n(s, &S.perm, C)) || (rc = dalloc_n(s, &S.ninf, C)) || (rc = dalloc_n(s, &S.box, C)) ||
        (rc = dalloc_n(s, &S.src, C)) || (rc = dalloc_n(s, &S.count, nbox + 1)) ||
        (rc = dalloc_n(s, &S.start, nbox + 1)))
      return rc;
    S.max_tiles = scan_tiles_for(nbox + 1);
    if ((rc = dalloc_n(s, &S.tiles, S.max_tiles))) return rc;
    // every index a step can read is in range from the start (see the bounds in the kernels)
    CK(cudaMemsetAsync(S.count, 0, sizeof(unsigned) * (nbox + 1), s->stream));
    CK(cudaMemsetAsync(S.start, 0, sizeof(unsigned) * (nbox + 1), s->stream));
    CK(cudaMemsetAsync(S.perm, 0, sizeof(unsigned) * C, s->stream));
    CK(cudaMemsetAsync(S.src, 0, sizeof(uint2) * C, s->stream));
    CK(cudaMemsetAsync(S.ninf, 0, sizeof(unsigned) * C, s->stream));
    CK(cudaMemsetAsync(S.box, 0, sizeof(unsigned) * C, s->stream));
    s->gh->nbox = (unsigned)nbox;
    s->gh->nbox1 = (unsigned)nbox + 1;
  } else {
    // box capacity: given, else twice the first population's grid plus headroom for growth
    size_t boxcap = p.box_capacity;
    if (boxcap == 0) {
      double est = 1.0;
      if (n_first > 0) {
        double R = p.interaction_radius;
        if (!(R > 0.0)) {
          R = 0.0;
          for (size_t i = 0; i < n_first; ++i) R = std::max(R, (double)d[i]);
        }
        const double L = p.box_length > 0.0 ? p.box_length : R + p.skin;
        const double* c[3] = {x, y, z};
        for (int a = 0; a < 3; ++a) {
          double lo = c[a][0], hi = c[a][0];
          for (size_t i = 1; i < n_first; ++i) {
            lo = std::min(lo, c[a][i]);
            hi = std::max(hi, c[a][i]);
          }
          est *= (L > 0.0 ? std::floor((hi - lo) / L) : 0.0) + 1.0;
        }
      }
      double cap = 2.0 * est + (s->growth ? 4.0 : 1.0) * (double)C + 4096.0;
      boxcap = (size_t)std::min(cap, 4.0e9);
    }
    s->box_capacity = boxcap;
    MechBuffers& b = s->mb;
    if ((rc = dalloc_n(s, &b.pos.x, C)) || (rc = dalloc_n(s, &b.pos.y, C)) ||
        (rc = dalloc_n(s, &b.pos.z, C)) || (rc = dalloc_n(s, &b.sorted.x, C)) ||
        (rc = dalloc_n(s, &b.sorted.y, C)) || (rc = dalloc_n(s, &b.sorted.z, C)))
      return rc;
    for (int h = 0; h < 2; ++h) {
      if ((rc = dalloc_n(s, &b.attr[h].diam, C)) || (rc = dalloc_n(s, &b.attr[h].id, C))) return rc;
      if (s->growth && (rc = dalloc_n(s, &b.attr[h].vol, C))) return rc;
    }
    if ((rc = dalloc_n(s, &b.key, C)) || (rc = dalloc_n(s, &b.rank, C)) ||
        (rc = dalloc_n(s, &b.perm, C)) || (rc = dalloc_n(s, &b.skey, C)) ||
        (rc = dalloc_n(s, &b.nbr, C)) || (rc = dalloc_n(s, &b.count, boxcap + 1)) ||
        (rc = dalloc_n(s, &b.start, boxcap + 1)))
      return rc;
    if (s->mixed && (rc = dalloc_n(s, &b.p4, C))) return rc;
    if ((rc = dalloc_n(s, &b.pack, C))) return rc;
    b.pset[0] = b.pos;
    b.p4set[0] = b.p4;
    if (p.skin > 0.0) {
      if (C >= (1ull << 27)) return fail(s, BDM_EINVAL, "a neighbour-list skin supports up to 2^27 agents");
      if ((rc = dalloc_n(s, &b.list, (size_t)kListCap * ((C + 31) / 32 * 32))) || (rc = dalloc_n(s, &b.list_n, C)) ||
          (rc = dalloc_n(s, &b.disp, C)) || (rc = dalloc_n(s, &b.pset[1].x, C)) ||
          (rc = dalloc_n(s, &b.pset[1].y, C)) || (rc = dalloc_n(s, &b.pset[1].z, C)) ||
          (rc = dalloc_n(s, &b.p4set[1], C)))
        return rc;
      const size_t ngrp = (C + 31) / 32;
      if (p.skip_stationary && ((rc = dalloc_n(s, &b.wmoved[0], ngrp)) || (rc = dalloc_n(s, &b.wmoved[1], ngrp)) ||
                                (rc = dalloc_n(s, &b.wbounds, ngrp)) || (rc = dalloc_n(s, &b.wrows, 9 * ngrp)) ||
                                (rc = dalloc_n(s, &b.evl, ngrp))))
        return rc;
      b.wstride = ngrp;
      CK(cudaMemsetAsync(b.list_n, 0, sizeof(unsigned) * C, s->stream));
      CK(cudaMemsetAsync(b.disp, 0, sizeof(float) * C, s->stream));
    }
    b.max_tiles = scan_tiles_for(boxcap + 1);
    if ((rc = dalloc_n(s, &b.tiles[0], b.max_tiles))) return rc;
    if (s->growth || p.p_apoptosis > 0.0) {
      if ((rc = dalloc_n(s, &b.tiles[1], scan_tiles_for(C + 1))) ||
          (rc = dalloc_n(s, &b.flag, C + 1)) || (rc = dalloc_n(s, &b.drank, C + 1)))
        return rc;
    }
    CK(cudaMemsetAsync(b.count, 0, sizeof(unsigned) * (boxcap + 1), s->stream));
    CK(cudaMemsetAsync(b.nbr, 0, sizeof(unsigned) * C, s->stream));
    CK(cudaMemsetAsync(b.skey, 0, sizeof(unsigned) * C, s->stream));
    MechConsts& mc = s->mc;
    mc.dt = p.dt;
    mc.k = p.repulsion;
    mc.gamma = p.attraction;
    mc.cap = p.max_displacement;
    mc.dtf = (float)p.dt;
    mc.kf = (float)p.repulsion;
    mc.gammaf = (float)p.attraction;
    mc.capf = (float)p.max_displacement;
    mc.interaction_radius = p.interaction_radius;
    mc.box_length = p.box_length;
    mc.box_capacity = (unsigned)std::min<size_t>(boxcap, 0xFFFFFFF0ull);
    mc.capacity = (unsigned)C;
    mc.force_variant = p.force_variant;
    mc.skin = p.skin;
    mc.skin_half = (float)(0.5 * p.skin * (1.0 - 1e-5));
    mc.max_cadence = 64;
    mc.skip_stationary = p.skip_stationary ? 1 : 0;
    mc.mixed = s->mixed ? 1 : 0;
  }
  if (s->diffusion) {
    const size_t nv = (size_t)p.grid_n[0] * p.grid_n[1] * p.grid_n[2];
    for (int a = 0; a < 3; ++a) s->gdims[a] = p.grid_n[a];
    if ((rc = dalloc_n(s, &s->grid[0], nv)) || (rc = dalloc_n(s, &s->grid[1], nv)) ||
        (rc = dalloc_n(s, &s->partials, (size_t)ftcs_partials_needed(s->gdims))))
      return rc;
    CK(cudaMemsetAsync(s->grid[0], 0, nv * sizeof(float), s->stream));
    const double lam = (p.diffusion_coeff * p.dt_diffusion) / (p.voxel * p.voxel);
    s->lam = (float)lam;
    s->mu_dt = (float)(p.decay * p.dt_diffusion);
  }
  CK(cudaMemcpyAsync(s->g, s->gh, sizeof(DevGrid), cudaMemcpyHostToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  // launch geometry: grid-stride kernels sized to the SM count and the agent capacity
  const int stream_blocks = s->sms * 8;
  const size_t need = (C + kBlock - 1) / kBlock;
  s->blocks_stream = (int)std::max<size_t>(1, std::min<size_t>(need, stream_blocks));
  s->blocks_force = s->mixed ? s->sms * (p.skin > 0.0 ? force_skin_blocks_per_sm(false)
                                                      : force_mixed_blocks_per_sm(s->mc.force_variant))
                             : force_fp64_blocks(C, s->sms);
  s->blocks_walk = p.skin > 0.0 ? s->sms * force_skin_blocks_per_sm(true) : s->blocks_force;
  s->blocks_list = s->sms * list_build_blocks_per_sm();
  const size_t tiles = s->is_sir ? s->sb.max_tiles : s->mb.max_tiles;
  s->blocks_scan = (int)std::max<size_t>(1, std::min<size_t>(tiles, (size_t)s->sms * 4));
  s->allocated = true;
  return BDM_OK;
}

// ---- error polling ------------------------------------------------------------------------------
int decode_err(bdm_sim* s, unsigned e) {
  if (!e) return BDM_OK;
  s->poisoned = true;
  if (e & ERR_TIMEOUT) return fail(s, BDM_ETIMEOUT, "a bounded device-side wait timed out");
  if (e & ERR_GRID_OVERFLOW)
    return fail(s, BDM_ENOMEM, "grid needs more boxes than box_capacity (%zu)", s->box_capacity);
  if (e & ERR_CAPACITY)
    return fail(s, BDM_ENOMEM, "division would exceed the agent capacity (%zu)", s->capacity);
  if (e & ERR_RADIUS)
    return fail(s, BDM_ESTATE, "invalid grid: radius/box length or agent extent out of range (mixed "
                               "precision needs interaction_radius >= the largest diameter)");
  return fail(s, BDM_ESTATE, "device index check failed (error bits 0x%x)", e);
}

int poll_err(bdm_sim* s) {
  if (s->poisoned) return fail(s, BDM_ESTATE, "handle is in an error state: %s", s->err.c_str());
  if (s->err_pending && cudaEventQuery(s->err_event) == cudaSuccess) {
    s->err_pending = false;
    return decode_err(s, *s->err_pinned);
  }
  cudaGetLastError();
  return BDM_OK;
}

int arm_err_poll(bdm_sim* s) {
  if (s->capturing) return BDM_OK;
  CK(cudaMemcpyAsync(s->err_pinned, &s->g->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaEventRecord(s->err_event, s->stream));
  s->err_pending = true;
  return BDM_OK;
}

// ---- one step -------------------------------------------------------------------------------------
int enqueue_diffusion(bdm_sim* s) {
  float* src = s->grid[s->grid_cur];
  float* dst = s->grid[s->grid_cur ^ 1];
  RUN("ftcs", 2, launch_ftcs(s->stream, src, dst, s->gdims, s->lam, s->mu_dt, s->partials, s->g));
  s->grid_cur ^= 1;
  return BDM_OK;
}

// Point the current-position views at position set pos_cur (two sets only with a skin).
void point_current(bdm_sim* s) {
  MechBuffers& b = s->mb;
  if (!b.pset[1].x) return;
  b.pos.x = b.pset[s->pos_cur].x;
  b.pos.y = b.pset[s->pos_cur].y;
  b.pos.z = b.pset[s->pos_cur].z;
  b.p4 = b.p4set[s->pos_cur];
}

int enqueue_mech_step(bdm_sim* s) {
  cudaStream_t st = s->stream;
  const bdm_params& p = s->p;
  MechBuffers& b = s->mb;
  AgentArrays A = b.attr[s->attr_cur], B = b.attr[s->attr_cur ^ 1];
  DevGrid* g = s->g;
  const uint2 pkey = make_uint2((unsigned)(p.seed & 0xFFFFFFFFull), p.run_id);
  if (p.p_apoptosis > 0.0) {  // R14: deaths at step start; survivors to the other attribute buffer
    const unsigned long long thr = (unsigned long long)std::floor(p.p_apoptosis * 4294967296.0);
    RUN("apo_flag", 1, launch_apoptosis_flags(st, b, A, g, thr, pkey, s->blocks_stream));
    CK(cudaMemsetAsync(b.tiles[1], 0, sizeof(unsigned long long) * scan_tiles_for(s->capacity + 1), st));
    RUN("scan_apo", 1, launch_scan(st, b.flag, b.drank, &g->ndiv1, b.tiles[1], &g->scan_ctr[1], &g->err, 0,
                                   s->blocks_scan));
    RUN("apo_compact", 2, launch_apoptosis_compact(st, b, A, B, g, s->blocks_stream));
    s->attr_cur ^= 1;
    A = b.attr[s->attr_cur];
    B = b.attr[s->attr_cur ^ 1];
    s->bounds_fresh = false;
  }
  if (s->growth) {
    RUN("grow", 1, launch_grow(st, b, A, g, p.growth_volume, p.division_volume, s->blocks_stream));
    CK(cudaMemsetAsync(b.tiles[1], 0, sizeof(unsigned long long) * scan_tiles_for(s->capacity + 1), st));
    RUN("scan_div", 1, launch_scan(st, b.flag, b.drank, &g->ndiv1, b.tiles[1], &g->scan_ctr[1], &g->err, 0,
                                   s->blocks_scan));
    RUN("divide", 1, launch_divide(st, b, A, g, p.division_offset_frac, pkey, (unsigned)s->capacity,
                                   s->blocks_stream));
    s->bounds_fresh = false;
  }
  if (!s->bounds_fresh) {
    CK(cudaMemsetAsync(&g->acc_min[0], 0xFF, sizeof(g->acc_min), st));
    CK(cudaMemsetAsync(&g->acc_max[0], 0x00, sizeof(g->acc_max), st));
    CK(cudaMemsetAsync(&g->acc_maxdiam, 0x00, sizeof(unsigned), st));
    RUN("bounds", 1, launch_bounds(st, b, A, g, s->blocks_stream));
  }
  RUN("finalize", 1, launch_finalize(st, g, s->mc));
  CK(cudaMemsetAsync(b.tiles[0], 0, sizeof(unsigned long long) * b.max_tiles, st));
  // with a skin, finalize decides on the device whether this step rebuilds: the rebuild kernels
  // then see 0 agents / 0 boxes on list steps, and the two force kernels skip the other kind
  RUN("key_hist", 1, launch_key_hist(st, b, A.id, g, s->blocks_stream));
  RUN("scan_box", 1, launch_scan(st, b.count, b.start, &g->nbox1_sort, b.tiles[0], &g->scan_ctr[0], &g->err,
                                 1, s->blocks_scan));
  RUN("scatter", 1, launch_scatter(st, b, g, s->blocks_stream));
  RUN("gather", 1, launch_gather(st, b, A, B, g, s->mixed, s->mc.skin > 0.0, s->blocks_stream));
  if (s->mc.skin > 0.0) {
    RUN("attr_copy", 1, launch_attr_copy(st, B, A, g, s->blocks_stream));
    RUN("list_build", 1, launch_list_build(st, b, g, s->blocks_list));
    RUN("force_walk", 1, launch_force_skin(st, b, s->pos_cur, g, s->mc, true, s->blocks_walk));  // overflow only
    if (s->mc.skip_stationary) RUN("still_warps", 1, launch_still_warps(st, b, s->pos_cur, g, s->blocks_stream));
    RUN("force_list", 1, launch_force_skin(st, b, s->pos_cur, g, s->mc, false, s->blocks_force));
    s->pos_cur ^= 1;  // the force kernels wrote the step's result into the other position set
    point_current(s);
    s->bounds_fresh = true;  // attributes stay in A
  } else {
    RUN(s->mixed ? "force_mixed" : "force_fp64", 1, launch_force(st, b, B, g, s->mc, s->mixed, s->blocks_force));
    s->bounds_fresh = !s->growth;
    s->attr_cur ^= 1;
    if (p.brownian_sigma > 0.0) {  // R13: after the capped update; the fused bounds are then stale
      RUN("brownian", 1, launch_brownian(st, b, b.attr[s->attr_cur], g, p.brownian_sigma, pkey, !s->mixed,
                                         s->blocks_stream));
      s->bounds_fresh = false;
    }
    if (p.chemotaxis != 0.0 && s->diffusion) {  // R15: the step-start grid, before secretion
      RUN("chemotaxis", 1, launch_chemotaxis(st, b, g, s->grid[s->grid_cur], s->gdims, p.grid_origin,
                                             p.voxel, p.chemotaxis, s->blocks_stream));
      s->bounds_fresh = false;
    }
  }
  if (s->diffusion) {
    if (p.secretion != 0.0)
      RUN("secrete", 1, launch_secrete(st, b, g, s->grid[s->grid_cur], s->gdims, p.grid_origin, p.voxel,
                                       (float)p.secretion, s->blocks_stream));
    int rc = enqueue_diffusion(s);
    if (rc) return rc;
  }
  RUN("step_done", 1, launch_step_done(st, g));
  return BDM_OK;
}

int enqueue_sir_step(bdm_sim* s) {
  SirSingle S = s->sb;
  S.run.agent_n = (unsigned)s->n_host;
  RUN("sir_step", 5, launch_sir_step(s->stream, S, s->g, s->blocks_stream, s->blocks_scan));
  if (s->diffusion) return enqueue_diffusion(s);
  return BDM_OK;
}

int enqueue_steps(bdm_sim* s, int n, bool diffusion_only) {
  for (int i = 0; i < n; ++i) {
    int rc = diffusion_only ? enqueue_diffusion(s) : (s->is_sir ? enqueue_sir_step(s) : enqueue_mech_step(s));
    if (rc) return rc;
  }
  return BDM_OK;
}

int launch_steps(bdm_sim* s, int n, bool diffusion_only) {
  if (s->prof.on) return enqueue_steps(s, n, diffusion_only);
  const auto key = std::make_tuple(n, (int)diffusion_only, s->attr_cur, s->grid_cur,
                                   (int)s->bounds_fresh, s->is_sir ? s->n_host : (size_t)0, s->pos_cur);
  auto it = s->graphs.find(key);
  if (it == s->graphs.end()) {
    GraphEntry ge;
    const int a0 = s->attr_cur, g0 = s->grid_cur, p0 = s->pos_cur;
    const bool f0 = s->bounds_fresh;
    CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    s->capturing = true;
    s->capture_kernels = 0;
    int rc = enqueue_steps(s, n, diffusion_only);
    s->capturing = false;
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(s->stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ce != cudaSuccess) return fail(s, BDM_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(s, BDM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
    ge.kernels = s->capture_kernels;
    ge.attr_cur = s->attr_cur;
    ge.grid_cur = s->grid_cur;
    ge.bounds_fresh = s->bounds_fresh;
    ge.pos_cur = s->pos_cur;
    s->attr_cur = a0;
    s->grid_cur = g0;
    s->bounds_fresh = f0;
    s->pos_cur = p0;
    point_current(s);
    if (s->graphs.size() > 64) {
      for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second.exec);
      s->graphs.clear();
    }
    it = s->graphs.emplace(key, ge).first;
  }
  CK(cudaGraphLaunch(it->second.exec, s->stream));
  g_launches += it->second.kernels;
  s->attr_cur = it->second.attr_cur;
  s->grid_cur = it->second.grid_cur;
  s->bounds_fresh = it->second.bounds_fresh;
  s->pos_cur = it->second.pos_cur;
  point_current(s);
  return BDM_OK;
}

int sync_read(bdm_sim* s) {
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaMemcpy(s->gh, s->g, sizeof(DevGrid), cudaMemcpyDeviceToHost));
  s->err_pending = false;
  if (!s->is_sir) s->n_host = s->gh->n;
  return decode_err(s, s->gh->err);
}

int ensure_allocated(bdm_sim* s) {
  if (s->allocated) return BDM_OK;
  return allocate(s, 0, nullptr, nullptr, nullptr, nullptr);
}

}  // namespace

// =================================================================================================
extern "C" {

int bdm_create(const bdm_params* p, bdm_sim** out) {
  if (!out) return BDM_EINVAL;
  *out = nullptr;
  bdm_sim* s = new (std::nothrow) bdm_sim();
  if (!s) return BDM_ENOMEM;
  int rc = check_params(s, p);
  if (rc) {
    // keep the handle so that bdm_last_error can explain the failure
    *out = s;
    s->poisoned = true;
    return rc;
  }
  s->p = *p;
  s->is_sir = p->kind == BDM_SIR;
  s->mixed = !s->is_sir && p->precision == BDM_MIXED;
  s->growth = !s->is_sir && p->growth_enabled;
  s->diffusion = p->diffusion_enabled != 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    *out = s;
    s->poisoned = true;
    return fail(s, BDM_ECUDA, "no CUDA device available");
  }
  if (p->stream) {
    s->stream = (cudaStream_t)p->stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      *out = s;
      s->poisoned = true;
      return fail(s, BDM_ECUDA, "cudaStreamCreate failed");
    }
    s->own_stream = true;
  }
  *out = s;
  if (p->capacity > 0 && !s->is_sir && p->box_capacity > 0) return allocate(s, 0, nullptr, nullptr, nullptr, nullptr);
  return BDM_OK;
}

int bdm_add_agents(bdm_sim* s, size_t n, const double* x, const double* y, const double* z, const float* diameter,
                   const double* volume, const uint8_t* sir_state) {
  if (!s) return BDM_EINVAL;
  int rc = poll_err(s);
  if (rc) return rc;
  if (n == 0) return BDM_OK;
  if (!x || !y || !z) return fail(s, BDM_EINVAL, "positions are NULL");
  if (!s->is_sir && !diameter) return fail(s, BDM_EINVAL, "diameter is NULL");
  if (!s->allocated) {
    rc = allocate(s, n, x, y, z, diameter);
    if (rc) return rc;
  }
  if (s->growth || !s->is_sir) {
    rc = sync_read(s);
    if (rc) return rc;
  }
  const size_t n0 = s->n_host;
  if (n0 + n > s->capacity) return fail(s, BDM_ENOMEM, "%zu agents exceed capacity %zu", n0 + n, s->capacity);
  cudaStream_t st = s->stream;
  if (s->is_sir) {
    const SirRun& r = s->sb.run;
    std::vector<int> q(3 * n);
    for (size_t i = 0; i < n; ++i) {
      const double v[3] = {x[i], y[i], z[i]};
      for (int a = 0; a < 3; ++a) {
        const double u = std::nearbyint(v[a] * 1024.0);
        if (!(u >= 0.0) || u >= (double)r.L)
          return fail(s, BDM_EINVAL, "agent %zu lies outside [0, sir_domain)", i);
        q[a * n + i] = (int)u;
      }
    }
    if (sir_state)
      for (size_t i = 0; i < n; ++i)
        if (sir_state[i] > 2) return fail(s, BDM_EINVAL, "sir_state must be 0, 1 or 2");
    const SirState& S = s->sb.a;
    CK(cudaMemcpyAsync(S.X + n0, q.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S.Y + n0, q.data() + n, n * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S.Z + n0, q.data() + 2 * n, n * sizeof(int), cudaMemcpyHostToDevice, st));
    if (sir_state) CK(cudaMemcpyAsync(S.st + n0, sir_state, n, cudaMemcpyHostToDevice, st));
    else CK(cudaMemsetAsync(S.st + n0, 0, n, st));
    // boxes, ranks and histogram entries of the new agents for the coming step
    RUN("sir_init", 1, launch_sir_init(st, s->sb, (unsigned)n0, (unsigned)(n0 + n), s->blocks_stream));
    s->n_host = n0 + n;
    CK(cudaStreamSynchronize(st));
    return BDM_OK;
  }
  MechBuffers& b = s->mb;
  const AgentArrays& A = b.attr[s->attr_cur];
  CK(cudaMemcpyAsync(b.pos.x + n0, x, n * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(b.pos.y + n0, y, n * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(b.pos.z + n0, z, n * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(A.diam + n0, diameter, n * sizeof(float), cudaMemcpyHostToDevice, st));
  if (s->growth && volume)
    CK(cudaMemcpyAsync(A.vol + n0, volume, n * sizeof(double), cudaMemcpyHostToDevice, st));
  // validation, ids, derived volumes and cleared outputs on the device; the count is committed only
  // once the upload has been checked
  CK(cudaMemsetAsync(&s->g->bad_input, 0xFF, sizeof(unsigned), st));
  RUN("prepare", 1, launch_prepare_agents(st, (unsigned)n0, (unsigned)n, b.pos.x, b.pos.y, b.pos.z, A.diam, A.id,
                                          A.vol, s->growth && !volume, b.nbr, b.skey, s->g, s->blocks_stream));
  CK(cudaMemcpyAsync(&s->gh->bad_input, &s->g->bad_input, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (s->gh->bad_input != 0xFFFFFFFFu)
    return fail(s, BDM_EINVAL, "agent %u: diameter must be > 0 and |position| < 1e9", s->gh->bad_input);
  s->n_stage = (unsigned)(n0 + n);
  CK(cudaMemcpyAsync(&s->g->n, &s->n_stage, sizeof(unsigned), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(&s->g->list_valid, 0, sizeof(unsigned), st));  // the next step rebuilds
  s->n_host = n0 + n;
  s->bounds_fresh = false;
  CK(cudaStreamSynchronize(st));
  return BDM_OK;
}

int bdm_set_grid(bdm_sim* s, const float* values) {
  if (!s) return BDM_EINVAL;
  int rc = poll_err(s);
  if (rc) return rc;
  if (!s->diffusion) return fail(s, BDM_EINVAL, "diffusion is not enabled");
  if (!values) return fail(s, BDM_EINVAL, "values is NULL");
  if ((rc = ensure_allocated(s))) return rc;
  const size_t nv = (size_t)s->gdims[0] * s->gdims[1] * s->gdims[2];
  CK(cudaMemcpyAsync(s->grid[s->grid_cur], values, nv * sizeof(float), cudaMemcpyHostToDevice, s->stream));
  RUN("grid_mass", 2, launch_grid_mass(s->stream, s->grid[s->grid_cur], s->gdims, s->partials, s->g));
  CK(cudaStreamSynchronize(s->stream));
  return BDM_OK;
}

int bdm_set_step(bdm_sim* s, uint64_t step) {
  if (!s) return BDM_EINVAL;
  int rc = poll_err(s);
  if (rc) return rc;
  if ((rc = ensure_allocated(s))) return rc;
  s->gh->step = step;
  CK(cudaMemcpyAsync(&s->g->step, &s->gh->step, sizeof(unsigned long long), cudaMemcpyHostToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return BDM_OK;
}

int bdm_reset(bdm_sim* s) {
  if (!s) return BDM_EINVAL;
  if (!s->allocated) return BDM_OK;
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaMemcpy(s->gh, s->g, sizeof(DevGrid), cudaMemcpyDeviceToHost));
  s->gh->n = 0;
  s->gh->step = 0;
  s->gh->err = 0;
  s->gh->sir_counts[0] = s->gh->sir_counts[1] = s->gh->sir_counts[2] = 0;
  s->gh->sir_sources = 0;
  s->gh->list_valid = 0;
  s->gh->rebuilds = 0;
  s->gh->skipped = 0;
  CK(cudaMemcpy(s->g, s->gh, sizeof(DevGrid), cudaMemcpyHostToDevice));
  // the SIR box histogram already holds the removed agents for their next step
  if (s->is_sir) CK(cudaMemset(s->sb.count, 0, sizeof(unsigned) * (s->box_capacity + 1)));
  s->n_host = 0;
  s->poisoned = false;
  s->err_pending = false;
  s->bounds_fresh = false;
  return BDM_OK;
}

int bdm_step(bdm_sim* s, int n) {
  if (!s) return BDM_EINVAL;
  int rc = poll_err(s);
  if (rc) return rc;
  if (n < 0) return fail(s, BDM_EINVAL, "negative step count");
  if (n == 0) return BDM_OK;
  if ((rc = ensure_allocated(s))) return rc;
  if (s->is_sir && s->n_host == 0 && !s->diffusion) return BDM_OK;
  rc = launch_steps(s, n, false);
  if (rc) return rc;
  return arm_err_poll(s);
}

int bdm_diffusion_step(bdm_sim* s, int n) {
  if (!s) return BDM_EINVAL;
  int rc = poll_err(s);
  if (rc) return rc;
  if (!s->diffusion) return fail(s, BDM_EINVAL, "diffusion is not enabled");
  if (n < 0) return fail(s, BDM_EINVAL, "negative step count");
  if (n == 0) return BDM_OK;
  if ((rc = ensure_allocated(s))) return rc;
  rc = launch_steps(s, n, true);
  if (rc) return rc;
  return arm_err_poll(s);
}

int bdm_get_state(bdm_sim* s, bdm_state* st) {
  if (!s || !st) return BDM_EINVAL;
  if (st->struct_size != sizeof(bdm_state))
    return fail(s, BDM_EINVAL, "state.struct_size %u != sizeof(bdm_state) %zu", st->struct_size, sizeof(bdm_state));
  if (s->poisoned) return fail(s, BDM_ESTATE, "handle is in an error state: %s", s->err.c_str());
  if (!s->allocated) {
    st->n = 0;
    st->step = 0;
    st->mass_total = 0.0;
    return BDM_OK;
  }
  int rc = sync_read(s);
  if (rc) return rc;
  const DevGrid& G = *s->gh;
  const size_t n = s->is_sir ? s->n_host : G.n;
  st->n = n;
  st->step = G.step;
  st->mass_total = G.mass;
  for (int k = 0; k < 3; ++k) {
    st->sir_counts[k] = G.sir_counts[k];
    st->grid_origin_q[k] = G.O[k];
    st->grid_dims[k] = G.dims[k];
  }
  st->grid_box_q = G.Lq;
  st->grid_rebuilds = G.rebuilds;
  st->list_entries = G.list_entries;
  st->stationary_skipped = G.skipped;
  cudaStream_t sm = s->stream;
  if (s->is_sir) {
    const SirState& S = s->sb.a;
    if (n && (st->x || st->y || st->z)) {
      std::vector<int> q(n);
      int* src[3] = {S.X, S.Y, S.Z};
      double* dst[3] = {st->x, st->y, st->z};
      for (int a = 0; a < 3; ++a) {
        if (!dst[a]) continue;
        CK(cudaMemcpy(q.data(), src[a], n * sizeof(int), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) dst[a][i] = (double)q[i] / 1024.0;
      }
    }
    if (n && st->sir_state) CK(cudaMemcpy(st->sir_state, S.st, n, cudaMemcpyDeviceToHost));
    if (n && st->neighbour_count) CK(cudaMemcpy(st->neighbour_count, s->sb.ninf, n * sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (n && st->box_id) CK(cudaMemcpy(st->box_id, s->sb.box, n * sizeof(unsigned), cudaMemcpyDeviceToHost));
  } else if (n && (st->x || st->y || st->z || st->diameter || st->volume || st->neighbour_count || st->box_id)) {
    MechBuffers& b = s->mb;
    const AgentArrays A = b.attr[s->attr_cur];
    double* ovol = (s->growth && st->volume) ? b.attr[s->attr_cur ^ 1].vol : nullptr;
    float* odiam = st->diameter ? (float*)b.perm : nullptr;
    unsigned* onbr = st->neighbour_count ? b.key : nullptr;
    unsigned* obox = st->box_id ? b.rank : nullptr;
    const bool pos = st->x || st->y || st->z;
    if (obox && b.pset[1].x)  // skin: a list step's box ids come from its step-start centres
      RUN("readout_box", 1, launch_readout_box(sm, b.pset[s->pos_cur ^ 1], b.skey, s->g, s->blocks_stream));
    if (odiam || ovol || onbr || obox)
      RUN("unsort", 1, launch_unsort(sm, b, A, s->g, nullptr, nullptr, nullptr, odiam, ovol, onbr, obox,
                                     s->blocks_stream));
    if (pos) {
      // each coordinate is permuted into id order, then copied to the host on a second stream
      // while the next one is permuted
      if (!s->copy_stream) {
        CK(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking));
        for (int a = 0; a < 3; ++a) CK(cudaEventCreateWithFlags(&s->axis_done[a], cudaEventDisableTiming));
      }
      const double* src[3] = {b.pos.x, b.pos.y, b.pos.z};
      double* stage[3] = {b.sorted.x, b.sorted.y, b.sorted.z};
      double* dst[3] = {st->x, st->y, st->z};
      for (int a = 0; a < 3; ++a) {
        if (!dst[a]) continue;
        RUN("unsort_axis", 1, launch_unsort_axis(sm, src[a], A.id, stage[a], s->g, s->blocks_stream));
        CK(cudaEventRecord(s->axis_done[a], sm));
        CK(cudaStreamWaitEvent(s->copy_stream, s->axis_done[a], 0));
        CK(cudaMemcpyAsync(dst[a], stage[a], n * sizeof(double), cudaMemcpyDeviceToHost, s->copy_stream));
      }
    }
    if (odiam) CK(cudaMemcpyAsync(st->diameter, odiam, n * sizeof(float), cudaMemcpyDeviceToHost, sm));
    if (ovol) CK(cudaMemcpyAsync(st->volume, ovol, n * sizeof(double), cudaMemcpyDeviceToHost, sm));
    if (onbr) CK(cudaMemcpyAsync(st->neighbour_count, onbr, n * sizeof(unsigned), cudaMemcpyDeviceToHost, sm));
    if (obox) CK(cudaMemcpyAsync(st->box_id, obox, n * sizeof(unsigned), cudaMemcpyDeviceToHost, sm));
    CK(cudaStreamSynchronize(sm));
    if (pos) CK(cudaStreamSynchronize(s->copy_stream));
    CK(cudaMemcpy(s->gh, s->g, sizeof(DevGrid), cudaMemcpyDeviceToHost));
    if ((rc = decode_err(s, s->gh->err))) return rc;
  }
  if (st->grid && s->diffusion) {
    const size_t nv = (size_t)s->gdims[0] * s->gdims[1] * s->gdims[2];
    CK(cudaMemcpyAsync(st->grid, s->grid[s->grid_cur], nv * sizeof(float), cudaMemcpyDeviceToHost, sm));
    CK(cudaStreamSynchronize(sm));
  }
  return BDM_OK;
}

void bdm_destroy(bdm_sim* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  s->prof.resolve();
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second.exec);
  for (void* q : s->allocs) {
    if (s->p.free) s->p.free(q, s->p.alloc_user);
    else cudaFree(q);
  }
  if (s->gh) cudaFreeHost(s->gh);
  if (s->err_pinned) cudaFreeHost(s->err_pinned);
  if (s->err_event) cudaEventDestroy(s->err_event);
  for (int a = 0; a < 3; ++a)
    if (s->axis_done[a]) cudaEventDestroy(s->axis_done[a]);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  cudaGetLastError();
  delete s;
}

const char* bdm_last_error(const bdm_sim* s) { return s ? s->err.c_str() : "NULL handle"; }

int bdm_profile(bdm_sim* s, int enable) {
  if (!s) return BDM_EINVAL;
  if (s->stream) CK(cudaStreamSynchronize(s->stream));
  s->prof.resolve();
  s->prof.stats.clear();
  s->prof.on = enable != 0;
  return BDM_OK;
}

int bdm_kernel_times(bdm_sim* s, bdm_kernel_time* out, int max, int* count) {
  if (!s) return BDM_EINVAL;
  if (s->stream) CK(cudaStreamSynchronize(s->stream));
  s->prof.resolve();
  const int m = (int)s->prof.stats.size();
  if (count) *count = m;
  for (int i = 0; i < m && i < max && out; ++i) {
    std::memset(out[i].name, 0, sizeof(out[i].name));
    std::strncpy(out[i].name, s->prof.stats[i].name.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = s->prof.stats[i].launches;
    out[i].total_ms = s->prof.stats[i].total_ms;
  }
  return BDM_OK;
}

uint64_t bdm_launch_count(void) { return g_launches.load(); }

const char* bdm_version(void) { return "bdm-gb300 1.0 (sm_103a)"; }

int bdm_philox(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  if (n == 0) return BDM_OK;
  if (!ctr || !key || !out || n > 0xFFFFFFFFull) return BDM_EINVAL;
  void *dc = nullptr, *dk = nullptr, *dout = nullptr;
  int rc = BDM_OK;
  if (cudaMalloc(&dc, n * 16) != cudaSuccess || cudaMalloc(&dk, n * 8) != cudaSuccess ||
      cudaMalloc(&dout, n * 16) != cudaSuccess) {
    rc = BDM_ENOMEM;
  } else if (cudaMemcpy(dc, ctr, n * 16, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(dk, key, n * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = BDM_ECUDA;
  } else {
    launch_philox(0, (unsigned)n, (const uint4*)dc, (const uint2*)dk, (uint4*)dout);
    g_launches += 1;
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(out, dout, n * 16, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = BDM_ECUDA;
  }
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  cudaGetLastError();
  return rc;
}

}  // extern "C"
