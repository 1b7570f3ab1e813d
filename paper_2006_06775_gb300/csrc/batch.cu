// batch.cu -- many SIR simulations advanced together, one persistent launch per step (C ABI in
// include/bdm.h, "Batched SIR ensemble").
//
// The runs keep their own parameters (BioDynaMo, arXiv 2006.06775, Sec. "Epidemiology use case":
// infection radius and probability, recovery probability, movement bound) and their own agents, in
// concatenated arrays with per-run offsets.  When every run's boxes and counts fit in a CTA's shared
// memory, a step is one CTA per run whose phases (histogram, scan, box order and infected list, push
// of infected agents into their neighbours' counts, update) are separated by __syncthreads.
// Otherwise a work list of (run, 256-agent tile) pairs lets one persistent grid cover every run, its
// phases separated by a grid barrier whose waits are bounded.  Every run computes exactly what it
// would compute alone: the arithmetic is integer and per run.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "bdm.h"
#include "common.cuh"
#include "sir.cuh"

using namespace bdm;

struct bdm_batch {
  std::vector<bdm_params> params;
  std::vector<std::vector<int>> hX, hY, hZ;       // staged agents per run (lattice units)
  std::vector<std::vector<unsigned char>> hS;
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool built = false, poisoned = false;
  int blocks = 0;
  bool cooperative = true;
  unsigned spin_limit = kSpinLimit;
  unsigned barrier_extra = 0;  // test hook: arrivals the grid barrier waits for beyond the grid
  bool persistent_only = false;
  size_t runs_smem = 0;        // > 0: one CTA per run with this much dynamic shared memory
  unsigned hist_len = 1024;
  std::vector<void*> allocs;
  std::vector<SirRun> runs;
  SirBatchDev dev{};
  DevGrid* g = nullptr;
  DevGrid* gh = nullptr;
  // n-step graphs; every step uses the same buffers, so one graph per n serves every starting step
  std::map<int, cudaGraphExec_t> graphs;
  unsigned long long steps_done = 0;
  void* (*alloc)(size_t, void*) = nullptr;
  void (*free)(void*, void*) = nullptr;
  void* alloc_user = nullptr;
};

extern "C" uint64_t bdm_launch_count(void);
void bdm_count_launches(unsigned long long k);  // api.cu

namespace {

int bfail(bdm_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  return code;
}

#define BCK(call)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return bfail(b, BDM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

int balloc(bdm_batch* b, void** p, size_t bytes) {
  bytes = std::max<size_t>(256, (bytes + 255) & ~size_t(255));
  void* q = nullptr;
  if (b->alloc) q = b->alloc(bytes, b->alloc_user);
  else if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    q = nullptr;
  }
  if (!q) return bfail(b, BDM_ENOMEM, "device allocation of %zu bytes failed", bytes);
  b->allocs.push_back(q);
  *p = q;
  return BDM_OK;
}
template <typename T>
int balloc_n(bdm_batch* b, T** p, size_t n) {
  return balloc(b, (void**)p, n * sizeof(T));
}

int build(bdm_batch* b) {
  const int R = (int)b->params.size();
  size_t total = 0, boxes = 0;
  std::vector<unsigned> tile_run, tile_start;
  b->runs.resize(R);
  for (int k = 0; k < R; ++k) {
    const bdm_params& p = b->params[k];
    const size_t n = b->hX[k].size();
    const int nb = sir_box_count(std::llrint(p.sir_domain * 1024.0), std::llrint(p.sir_radius * 1024.0),
                                 p.sir_boxes, n);
    const long long L = std::llrint(p.sir_domain * 1024.0), r = std::llrint(p.sir_radius * 1024.0);
    if (L % nb != 0 || L / nb < r)
      return bfail(b, BDM_EINVAL, "run %d: sir_boxes %d must divide the lattice side with box >= r", k, nb);
    SirRun& s = b->runs[k];
    s.L = (int)L;
    s.nb = nb;
    s.Lb = (int)(L / nb);
    s.invLb = 1.0f / (float)s.Lb;
    s.s = (int)std::llrint(p.sir_step * 1024.0);
    s.span = 2ull * (unsigned long long)s.s + 1ull;
    s.r2 = r * r;
    s.thr_inf = (unsigned long long)std::floor(p.p_infect * 4294967296.0);
    s.thr_rec = (unsigned long long)std::floor(p.p_recover * 4294967296.0);
    s.key = make_uint2((unsigned)(p.seed & 0xFFFFFFFFull), p.run_id);
    s.agent_off = (unsigned)total;
    s.agent_n = (unsigned)n;
    s.box_off = (unsigned)boxes;
    for (size_t t = 0; t < n; t += kBlock) {
      tile_run.push_back((unsigned)k);
      tile_start.push_back((unsigned)(total + t));
    }
    total += n;
    boxes += (size_t)nb * nb * nb;
    if (total > 0xF0000000ull || boxes > 0xF0000000ull)
      return bfail(b, BDM_EINVAL, "batch too large for 32-bit indices");
  }
  SirBatchDev& D = b->dev;
  const size_t A = std::max<size_t>(total, 1);
  int rc;
  if ((rc = balloc_n(b, &D.a.X, A)) || (rc = balloc_n(b, &D.a.Y, A)) || (rc = balloc_n(b, &D.a.Z, A)) ||
      (rc = balloc_n(b, &D.a.st, A)))
    return rc;
  D.max_tiles = (unsigned)((boxes + 1 + kScanTile - 1) / kScanTile + 1);
  SirRun* druns = nullptr;
  unsigned *dtr = nullptr, *dts = nullptr;
  if ((rc = balloc_n(b, &D.kn, A)) || (rc = balloc_n(b, &D.rk, A)) ||
      (rc = balloc_n(b, &D.perm, A)) || (rc = balloc_n(b, &D.ninf, A)) ||
      (rc = balloc_n(b, &D.box, A)) || (rc = balloc_n(b, &D.src, A)) ||
      (rc = balloc_n(b, &D.count, boxes + 1)) || (rc = balloc_n(b, &D.start, boxes + 1)) ||
      (rc = balloc_n(b, &D.tiles, D.max_tiles)) || (rc = balloc_n(b, &druns, (size_t)R)) ||
      (rc = balloc_n(b, &dtr, std::max<size_t>(tile_run.size(), 1))) ||
      (rc = balloc_n(b, &dts, std::max<size_t>(tile_start.size(), 1))) ||
      (rc = balloc_n(b, &D.hist, (size_t)b->hist_len * R * 3)) || (rc = balloc_n(b, &D.bar, 2)) ||
      (rc = balloc_n(b, &b->g, 1)))
    return rc;
  cudaStream_t s = b->stream;
  for (int k = 0; k < R; ++k) {
    const size_t n = b->hX[k].size(), off = b->runs[k].agent_off;
    if (!n) continue;
    BCK(cudaMemcpyAsync(D.a.X + off, b->hX[k].data(), n * 4, cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(D.a.Y + off, b->hY[k].data(), n * 4, cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(D.a.Z + off, b->hZ[k].data(), n * 4, cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(D.a.st + off, b->hS[k].data(), n, cudaMemcpyHostToDevice, s));
  }
  BCK(cudaMemcpyAsync(druns, b->runs.data(), sizeof(SirRun) * R, cudaMemcpyHostToDevice, s));
  if (!tile_run.empty()) {
    BCK(cudaMemcpyAsync(dtr, tile_run.data(), 4 * tile_run.size(), cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(dts, tile_start.data(), 4 * tile_start.size(), cudaMemcpyHostToDevice, s));
  }
  // start/perm/src are zeroed so that every index a step can read is in range even when a bounded
  // barrier wait gives up before the phase that writes them has finished
  // the first step's scan needs clear tile flags; later steps clear them after their own scan
  BCK(cudaMemsetAsync(D.tiles, 0, sizeof(unsigned long long) * D.max_tiles, s));
  BCK(cudaMemsetAsync(D.count, 0, 4 * (boxes + 1), s));
  BCK(cudaMemsetAsync(D.start, 0, 4 * (boxes + 1), s));
  BCK(cudaMemsetAsync(D.perm, 0, 4 * A, s));
  BCK(cudaMemsetAsync(D.src, 0, 8 * A, s));
  BCK(cudaMemsetAsync(D.ninf, 0, 4 * A, s));
  BCK(cudaMemsetAsync(D.hist, 0, 4 * (size_t)b->hist_len * R * 3, s));
  BCK(cudaMemsetAsync(D.bar, 0, 8, s));
  BCK(cudaMallocHost((void**)&b->gh, sizeof(DevGrid)));
  std::memset(b->gh, 0, sizeof(DevGrid));
  BCK(cudaMemcpyAsync(b->g, b->gh, sizeof(DevGrid), cudaMemcpyHostToDevice, s));
  D.run = druns;
  D.tile_run = dtr;
  D.tile_start = dts;
  D.ntiles = (unsigned)tile_run.size();
  D.runs = (unsigned)R;
  D.total_agents = (unsigned)total;
  D.total_boxes = (unsigned)boxes;
  D.hist_len = b->hist_len;
  int sms = 0, dev = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = sir_ensemble_blocks_per_sm();
  if (per_sm < 1) return bfail(b, BDM_ECUDA, "persistent SIR kernel cannot be resident");
  b->blocks = sms * per_sm;
  // one CTA per run when every run's boxes and counts fit in a CTA's shared memory (the grid-barrier
  // test hook needs the persistent kernel)
  if (!b->persistent_only && b->barrier_extra == 0) {
    size_t words = 0;
    for (const SirRun& r : b->runs)
      words = std::max(words, (size_t)r.nb * r.nb * r.nb + 1 + r.agent_n);
    b->runs_smem = sir_runs_smem_bytes(words);
    cudaGetLastError();
  }
  // boxes, ranks and histogram of the first step
  launch_sir_init_batch(s, D, b->blocks);
  BCK(cudaGetLastError());
  bdm_count_launches(1);
  BCK(cudaStreamSynchronize(s));
  b->built = true;
  return BDM_OK;
}

int enqueue(bdm_batch* b, int n) {
  if (b->runs_smem) {
    for (int i = 0; i < n; ++i) launch_sir_runs(b->stream, b->dev, b->g, b->runs_smem);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(b, BDM_ECUDA, "per-run SIR launch failed: %s", cudaGetErrorString(e));
    return BDM_OK;
  }
  for (int i = 0; i < n; ++i) {
    cudaError_t e = launch_sir_ensemble(b->stream, b->dev, b->g, b->blocks, b->barrier_extra,
                                        b->spin_limit, b->cooperative);
    if (e != cudaSuccess) return bfail(b, BDM_ECUDA, "persistent SIR launch failed: %s", cudaGetErrorString(e));
  }
  return BDM_OK;
}

}  // namespace

extern "C" {

int bdm_batch_create(const bdm_params* per_sim, int count, const bdm_batch_options* opt, bdm_batch** out) {
  if (!out) return BDM_EINVAL;
  *out = nullptr;
  bdm_batch* b = new (std::nothrow) bdm_batch();
  if (!b) return BDM_ENOMEM;
  *out = b;
  if (!per_sim || count <= 0) {
    b->poisoned = true;
    return bfail(b, BDM_EINVAL, "need at least one simulation");
  }
  for (int k = 0; k < count; ++k) {
    const bdm_params& p = per_sim[k];
    if (p.struct_size != sizeof(bdm_params) || p.kind != BDM_SIR) {
      b->poisoned = true;
      return bfail(b, BDM_EINVAL, "simulation %d: struct_size mismatch or kind is not BDM_SIR", k);
    }
    const double Lu = std::nearbyint(p.sir_domain * 1024.0);
    if (!(Lu >= 1.0) || Lu >= 2147483647.0 || !(p.sir_radius >= 0.0) || !(p.sir_step >= 0.0) ||
        std::nearbyint(p.sir_step * 1024.0) >= Lu || !(p.p_infect >= 0.0 && p.p_infect <= 1.0) ||
        !(p.p_recover >= 0.0 && p.p_recover <= 1.0) || p.sir_boxes < 0) {
      b->poisoned = true;
      return bfail(b, BDM_EINVAL, "simulation %d: invalid SIR parameters", k);
    }
  }
  b->params.assign(per_sim, per_sim + count);
  b->hX.resize(count);
  b->hY.resize(count);
  b->hZ.resize(count);
  b->hS.resize(count);
  if (opt) {
    if (opt->struct_size != sizeof(bdm_batch_options)) {
      b->poisoned = true;
      return bfail(b, BDM_EINVAL, "options.struct_size mismatch");
    }
    if (opt->history_steps > 0) b->hist_len = (unsigned)opt->history_steps;
    if (opt->spin_limit > 0) b->spin_limit = opt->spin_limit;
    b->barrier_extra = opt->barrier_extra;
    b->persistent_only = opt->persistent_only != 0;
    b->alloc = opt->alloc;
    b->free = opt->free;
    b->alloc_user = opt->alloc_user;
    b->stream = (cudaStream_t)opt->stream;
  }
  if (!b->stream) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      b->poisoned = true;
      return bfail(b, BDM_ECUDA, "cudaStreamCreate failed (no CUDA device?)");
    }
    b->own_stream = true;
  }
  return BDM_OK;
}

int bdm_batch_add_agents(bdm_batch* b, int sim, size_t n, const double* x, const double* y,
                         const double* z, const uint8_t* sir_state) {
  if (!b) return BDM_EINVAL;
  if (b->poisoned) return bfail(b, BDM_ESTATE, "batch is in an error state");
  if (b->built) return bfail(b, BDM_ESTATE, "agents must be added before the first step");
  if (sim < 0 || sim >= (int)b->params.size()) return bfail(b, BDM_EINVAL, "no simulation %d", sim);
  if (n && (!x || !y || !z)) return bfail(b, BDM_EINVAL, "positions are NULL");
  const double L = std::nearbyint(b->params[sim].sir_domain * 1024.0);
  for (size_t i = 0; i < n; ++i) {
    const double v[3] = {std::nearbyint(x[i] * 1024.0), std::nearbyint(y[i] * 1024.0),
                         std::nearbyint(z[i] * 1024.0)};
    for (int a = 0; a < 3; ++a)
      if (!(v[a] >= 0.0) || v[a] >= L) return bfail(b, BDM_EINVAL, "agent %zu lies outside the domain", i);
    b->hX[sim].push_back((int)v[0]);
    b->hY[sim].push_back((int)v[1]);
    b->hZ[sim].push_back((int)v[2]);
    const uint8_t st = sir_state ? sir_state[i] : 0;
    if (st > 2) return bfail(b, BDM_EINVAL, "sir_state must be 0, 1 or 2");
    b->hS[sim].push_back(st);
  }
  return BDM_OK;
}

int bdm_batch_step(bdm_batch* b, int n) {
  if (!b) return BDM_EINVAL;
  if (b->poisoned) return bfail(b, BDM_ESTATE, "batch is in an error state: %s", b->err.c_str());
  if (n < 0) return bfail(b, BDM_EINVAL, "negative step count");
  if (n == 0) return BDM_OK;
  if (!b->built) {
    int rc = build(b);
    if (rc) {
      b->poisoned = true;
      return rc;
    }
  }
  auto it = b->graphs.find(n);
  if (it == b->graphs.end()) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int rc = ok ? enqueue(b, n) : BDM_OK;
    if (ok) ok = cudaStreamEndCapture(b->stream, &graph) == cudaSuccess && rc == BDM_OK;
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
      // a cooperative launch that cannot be captured is issued step by step instead
      cudaGetLastError();
      rc = enqueue(b, n);
      if (rc) return rc;
      bdm_count_launches((unsigned long long)n * (b->runs_smem ? 2u : 1u));
      b->steps_done += (unsigned long long)n;
      return BDM_OK;
    }
    it = b->graphs.emplace(n, exec).first;
  }
  BCK(cudaGraphLaunch(it->second, b->stream));
  bdm_count_launches((unsigned long long)n * (b->runs_smem ? 2u : 1u));
  b->steps_done += (unsigned long long)n;
  return BDM_OK;
}

int bdm_batch_sync(bdm_batch* b) {
  if (!b) return BDM_EINVAL;
  if (!b->built) return BDM_OK;
  BCK(cudaStreamSynchronize(b->stream));
  BCK(cudaMemcpy(b->gh, b->g, sizeof(DevGrid), cudaMemcpyDeviceToHost));
  if (b->gh->err) {
    b->poisoned = true;
    if (b->gh->err & ERR_TIMEOUT) return bfail(b, BDM_ETIMEOUT, "a bounded grid-barrier wait timed out");
    return bfail(b, BDM_ESTATE, "device error bits 0x%x", b->gh->err);
  }
  return BDM_OK;
}

int bdm_batch_get_state(bdm_batch* b, int sim, bdm_state* st) {
  if (!b || !st) return BDM_EINVAL;
  if (st->struct_size != sizeof(bdm_state)) return bfail(b, BDM_EINVAL, "state.struct_size mismatch");
  if (sim < 0 || sim >= (int)b->params.size()) return bfail(b, BDM_EINVAL, "no simulation %d", sim);
  if (!b->built) {
    st->n = b->hX[sim].size();
    st->step = 0;
    return BDM_OK;
  }
  int rc = bdm_batch_sync(b);
  if (rc) return rc;
  const SirRun& r = b->runs[sim];
  const size_t n = r.agent_n, off = r.agent_off;
  const SirState& S = b->dev.a;
  st->n = n;
  st->step = b->gh->step;
  st->mass_total = 0.0;
  if (b->gh->step > 0) {
    const unsigned slot = (unsigned)((b->gh->step - 1) % b->hist_len);
    BCK(cudaMemcpy(st->sir_counts, b->dev.hist + ((size_t)slot * b->runs.size() + sim) * 3, 12,
                   cudaMemcpyDeviceToHost));
  } else {
    std::memset(st->sir_counts, 0, sizeof(st->sir_counts));
  }
  if (n && (st->x || st->y || st->z)) {
    std::vector<int> q(n);
    int* src[3] = {S.X, S.Y, S.Z};
    double* dst[3] = {st->x, st->y, st->z};
    for (int a = 0; a < 3; ++a) {
      if (!dst[a]) continue;
      BCK(cudaMemcpy(q.data(), src[a] + off, n * 4, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < n; ++i) dst[a][i] = (double)q[i] / 1024.0;
    }
  }
  if (n && st->sir_state) BCK(cudaMemcpy(st->sir_state, S.st + off, n, cudaMemcpyDeviceToHost));
  if (n && st->neighbour_count) BCK(cudaMemcpy(st->neighbour_count, b->dev.ninf + off, n * 4, cudaMemcpyDeviceToHost));
  if (n && st->box_id) {
    BCK(cudaMemcpy(st->box_id, b->dev.box + off, n * 4, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) st->box_id[i] -= r.box_off;  // run-local box id
  }
  return BDM_OK;
}

int bdm_batch_counts(bdm_batch* b, uint32_t* out, int max_steps, int* steps) {
  if (!b) return BDM_EINVAL;
  int rc = bdm_batch_sync(b);
  if (rc) return rc;
  const unsigned long long done = b->built ? b->gh->step : 0ull;
  const unsigned long long avail = std::min<unsigned long long>(done, b->hist_len);
  const int m = (int)std::min<unsigned long long>(avail, (unsigned long long)std::max(max_steps, 0));
  if (steps) *steps = m;
  const size_t R = b->params.size();
  std::vector<uint32_t> slot(R * 3);
  for (int k = 0; k < m; ++k) {  // the last m steps, oldest first
    const unsigned long long step = done - (unsigned long long)m + (unsigned long long)k;
    const unsigned s = (unsigned)(step % b->hist_len);
    BCK(cudaMemcpy(out + (size_t)k * R * 3, b->dev.hist + (size_t)s * R * 3, R * 3 * 4, cudaMemcpyDeviceToHost));
  }
  return BDM_OK;
}

void bdm_batch_destroy(bdm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (void* q : b->allocs) {
    if (b->free) b->free(q, b->alloc_user);
    else cudaFree(q);
  }
  if (b->gh) cudaFreeHost(b->gh);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  cudaGetLastError();
  delete b;
}

const char* bdm_batch_last_error(const bdm_batch* b) { return b ? b->err.c_str() : "NULL batch"; }

}  // extern "C"
