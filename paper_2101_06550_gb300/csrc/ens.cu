// Ensemble runtime: many Cahn-Hilliard simulations of uneven sizes advanced
// together (the batched pattern the thesis's 2D statistics rest on, Sec. 7.3.2:
// batches of simulations per domain size, run concurrently).
//
// Simulations that share (n, L) form a group: one ChGroup with packed
// device-resident state, C^n and C^{n-1} for `capacity` slots, and per-slot LHS
// factors, so a group mixes any gammas (one LHS per distinct matrix, as the
// thesis proposes for uneven batches).  Slots [0, active) of a group are
// stepped; the host keeps them packed (ens_slot_move).  The two state buffers
// of a group swap roles each step (no copy).
//
// FP32 + refinement ensembles advance every group with three launches per
// step, one per phase (right-hand side, x solves, y solves with the update):
// each launch is a persistent grid whose blocks stride over the work items of
// all groups, packed group after group in a tuned order (ens_tune_schedule
// picks the order, the blocks per SM of each phase and the y strips' width).
// FP64 ensembles launch each group's kernels on a branch of their own.
// ens_step replays a CUDA graph of two steps; an odd leftover step runs
// eagerly.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "chgroup.cuh"

using namespace chx;

namespace {


struct EnsGroup {
  ChGroup g;
  int n = 0, capacity = 0, active = 0;
  double l = 0, gamma = 0;
  double* d_state[2] = {nullptr, nullptr};  // each capacity * n * n doubles
  int cur = 0;                              // index of the buffer holding C^n
  void* d_work = nullptr;
  size_t work_bytes = 0, bytes = 0;
  cudaStream_t stream = nullptr;            // branch stream used during capture
  cudaEvent_t done = nullptr;
  std::vector<double> slot_gamma;           // gamma each slot is factorised for
  int* status = nullptr;                    // the ensemble's device status word
  bool live = false;
  // Cahn-Hilliard-Cook forcing (ens_group_set_cook): deviates of every slot,
  // drawn each step with the device step counter, then the forced step
  double sigma = 0;
  uint64_t seed = 0;
  double* d_rho = nullptr;                  // capacity * 2 * n * n doubles
  uint64_t* d_step = nullptr;
  size_t cook_bytes = 0;
};

}  // namespace

// The FP32 ensemble's packed schedule (see the file comment).
constexpr int kEnsMaxGroups = 256;  // groups the phase launches cover (more: per-group branches)
struct EnsSchedule {
  // tuned choices: order 0 = most work per item first, 1 = least first;
  // blocks per SM per phase (0 = as many as fit); points per work item of the
  // solves (the x rows / y columns of every group's tiles follow from it)
  int order_mode = 0, bps[3] = {0, 0, 0}, target = kFFTarget;
  // derived for the current groups and active counts
  int ngroups = 0, nitems[3] = {0, 0, 0}, blocks[3] = {0, 0, 0};
  size_t smem[3] = {0, 0, 0};
  bool valid = false;
  FFStep* d_steps = nullptr;  // kEnsMaxGroups
  int* d_order = nullptr;     // kEnsMaxGroups
  int* d_start = nullptr;     // 3 x (kEnsMaxGroups + 1)
  std::vector<EnsGroup*> members;  // groups in schedule order
};

struct chx_ens {
  PlanHdr hdr;
  int precision;
  double dt;
  size_t budget, used;
  std::vector<EnsGroup*>* groups;
  cudaGraphExec_t exec;
  bool dirty;  // active counts or groups changed since the graph was built
  cudaEvent_t fork;
  cudaStream_t cap;  // private stream the graph is captured on (never the legacy stream)
  EnsSchedule* sched;  // FP32 + refinement ensembles only
};

namespace {

size_t state_bytes(int n, int cap) { return 2 * (size_t)cap * n * n * sizeof(double); }

void free_group(EnsGroup* G) {
  if (!G) return;
  group_free(&G->g);
  cudaFree(G->d_state[0]);
  cudaFree(G->d_state[1]);
  cudaFree(G->d_work);
  cudaFree(G->d_rho);
  cudaFree(G->d_step);
  if (G->stream) cudaStreamDestroy(G->stream);
  if (G->done) cudaEventDestroy(G->done);
  delete G;
}

EnsGroup* get_group(chx_ens* e, int id) {
  if (!e || e->hdr.magic != kMagicEns || id < 0 || id >= (int)e->groups->size()) return nullptr;
  EnsGroup* G = (*e->groups)[id];
  return (G && G->live) ? G : nullptr;
}

void drop_graph(chx_ens* e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  e->exec = nullptr;
  e->dirty = true;
  if (e->sched) e->sched->valid = false;
}

bool packed(const chx_ens* e) { return e->precision == CHX_PREC_F32_REFINE && e->sched; }

// Lays out the packed FP32 schedule for the current groups and active counts
// and uploads it (synchronous; outside any capture).  Returns CHX_OK with
// valid = false when the groups do not fit the schedule (the per-group branches
// then step them).
int build_schedule(chx_ens* e) {
  EnsSchedule& S = *e->sched;
  S.valid = false;
  S.members.clear();
  for (EnsGroup* G : *e->groups)
    if (G && G->live && G->active > 0) S.members.push_back(G);
  S.ngroups = (int)S.members.size();
  if (S.ngroups == 0 || S.ngroups > kEnsMaxGroups) return CHX_OK;
  std::vector<FFStep> steps(S.ngroups);
  for (int k = 0; k < S.ngroups; ++k) {
    EnsGroup* G = S.members[k];
    G->g.noise = G->sigma > 0 ? G->d_rho : nullptr;
    steps[k] = ff_step_params(&G->g, G->active, G->d_state[0], G->d_state[1], G->d_work, S.target);
    steps[k].cur0 = G->cur;
    G->g.noise = nullptr;
    if (steps[k].xs < 1 || steps[k].ysc < 1) return CHX_OK;  // a tile does not fit: per-group launches
  }
  // order: most work per item first (largest grids), or least first
  std::vector<int> order(S.ngroups);
  for (int k = 0; k < S.ngroups; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return S.order_mode == 0 ? S.members[a]->n > S.members[b]->n : S.members[a]->n < S.members[b]->n;
  });
  std::vector<int> start(3 * (kEnsMaxGroups + 1), 0);
  bool noise = false;
  size_t sx = 0, sy = 0;
  for (int k = 0; k < S.ngroups; ++k) {
    const FFStep& P = steps[order[k]];
    for (int ph = 0; ph < 3; ++ph)
      start[ph * (kEnsMaxGroups + 1) + k + 1] = start[ph * (kEnsMaxGroups + 1) + k] + ens_phase_items(ph, P);
    noise = noise || P.noise;
    sx = std::max(sx, x_solve_smem(P.nx, P.ny, P.X.P, P.xs));
    sy = std::max(sy, y_solve_smem(P.ny, P.Y.P, P.ysc, P.yrb));
  }
  if (sx > ens_phase_smem_max() || sy > ens_phase_smem_max()) return CHX_OK;  // per-group launches
  int dev = 0, sms = 0;
  int rc = cuda_check(cudaGetDevice(&dev), "ens: device");
  if (!rc) rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "ens: SM count");
  if (rc) return rc;
  S.smem[0] = noise ? 1 : 0;
  S.smem[1] = sx;
  S.smem[2] = sy;
  for (int ph = 0; ph < 3; ++ph) {
    S.nitems[ph] = start[ph * (kEnsMaxGroups + 1) + S.ngroups];
    const int occ = ens_phase_occupancy(ph, S.smem[ph]);
    const int bps = S.bps[ph] > 0 && S.bps[ph] < occ ? S.bps[ph] : occ;
    S.blocks[ph] = std::min(S.nitems[ph], sms * bps);
  }
  std::vector<FFStep> packed_steps(S.ngroups);
  for (int k = 0; k < S.ngroups; ++k) packed_steps[k] = steps[k];
  if ((rc = cuda_check(cudaMemcpy(S.d_steps, packed_steps.data(), S.ngroups * sizeof(FFStep), cudaMemcpyHostToDevice),
                       "ens: schedule upload")) ||
      (rc = cuda_check(cudaMemcpy(S.d_order, order.data(), S.ngroups * sizeof(int), cudaMemcpyHostToDevice),
                       "ens: schedule upload")) ||
      (rc = cuda_check(cudaMemcpy(S.d_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice),
                       "ens: schedule upload")))
    return rc;
  S.valid = true;
  return CHX_OK;
}

// One packed FP32 step of every scheduled group at step parity q (C^n of a
// group in its buffer cur ^ q); Cook groups draw their deviates first.
void step_packed(chx_ens* e, int q, cudaStream_t st) {
  EnsSchedule& S = *e->sched;
  for (EnsGroup* G : S.members)
    if (G->sigma > 0) {
      launch_noise_normals(G->d_rho, G->n, G->n, G->active, G->seed, 0, 0, G->d_step, st);
    }
  for (int ph = 0; ph < 3; ++ph)
    launch_ens_phase_ff(ph, S.d_steps, S.d_order, S.d_start + ph * (kEnsMaxGroups + 1), S.ngroups, S.nitems[ph],
                        S.blocks[ph], q, S.smem[ph], st);
  for (EnsGroup* G : S.members)
    if (G->sigma > 0) launch_step_advance(G->d_step, st);
}

void step_group(EnsGroup* G, cudaStream_t st) {
  if (G->active < 1) return;
  if (G->sigma > 0) group_cook_deviates(&G->g, G->active, G->d_rho, G->seed, 0, 0, G->d_step, st);
  group_step(&G->g, G->active, G->d_state[G->cur], G->d_state[1 - G->cur], G->d_work, 0, st, nullptr, G->status);
  if (G->sigma > 0) {
    launch_step_advance(G->d_step, st);
    group_cook_clear(&G->g);
  }
  G->cur = 1 - G->cur;
}

// Two steps of every active group: the packed phase launches (FP32 +
// refinement), or each group on its own branch.  Captured on the ensemble's
// private stream; the instantiated graph can launch on any stream.
int build_graph(chx_ens* e) {
  drop_graph(e);
  if (packed(e)) {
    int rc0 = build_schedule(e);
    if (rc0) return rc0;
  }
  const bool use_packed = packed(e) && e->sched->valid;
  cudaGraph_t graph = nullptr;
  cudaStream_t st = e->cap;
  int rc = cuda_check(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "ens: begin capture");
  if (rc) return rc;
  std::vector<int> saved;
  if (use_packed) {
    step_packed(e, 0, st);
    step_packed(e, 1, st);
  } else {
    cudaEventRecord(e->fork, st);
    for (EnsGroup* G : *e->groups) {
      saved.push_back(G && G->live ? G->cur : 0);
      if (!G || !G->live || G->active < 1) continue;
      cudaStreamWaitEvent(G->stream, e->fork, 0);
      step_group(G, G->stream);
      step_group(G, G->stream);
      cudaEventRecord(G->done, G->stream);
      cudaStreamWaitEvent(st, G->done, 0);
    }
  }
  cudaError_t ce = cudaStreamEndCapture(st, &graph);
  // capture does not execute: put the role flags back (two flips cancel anyway)
  if (!use_packed)
    for (size_t k = 0; k < e->groups->size(); ++k)
      if ((*e->groups)[k] && (*e->groups)[k]->live) (*e->groups)[k]->cur = saved[k];
  rc = cuda_check(ce, "ens: end capture");
  if (!rc) rc = cuda_check(cudaGraphInstantiate(&e->exec, graph, 0), "ens: graph instantiate");
  if (graph) cudaGraphDestroy(graph);
  if (rc) {
    e->exec = nullptr;
    return rc;
  }
  e->dirty = false;
  return CHX_OK;
}

}  // namespace

namespace chx {
void ens_free(chx_ens* e) {
  if (!e) return;
  drop_graph(e);
  if (e->groups) {
    for (EnsGroup* G : *e->groups) free_group(G);
    delete e->groups;
  }
  if (e->fork) cudaEventDestroy(e->fork);
  if (e->cap) cudaStreamDestroy(e->cap);
  if (e->sched) {
    cudaFree(e->sched->d_steps);
    cudaFree(e->sched->d_order);
    cudaFree(e->sched->d_start);
    delete e->sched;
  }
  hdr_free(&e->hdr);
  free(e);
}
}  // namespace chx

extern "C" int ens_create(chx_ens** out, int precision, double dt, size_t hbm_budget_bytes) {
  if (!out) return fail(CHX_EINVAL, "ens_create: null pointer");
  *out = nullptr;
  if (precision != CHX_PREC_F64 && precision != CHX_PREC_F32_REFINE)
    return fail(CHX_EINVAL, "ens_create: precision %d", precision);
  if (!(dt > 0) || !isfinite(dt)) return fail(CHX_EINVAL, "ens_create: dt %g", dt);
  chx_ens* e = (chx_ens*)calloc(1, sizeof(chx_ens));
  if (!e) return fail(CHX_ENOMEM, "ens_create: allocation");
  int rc = hdr_init(&e->hdr, kMagicEns);
  e->precision = precision;
  e->dt = dt;
  e->budget = hbm_budget_bytes;
  e->groups = new std::vector<EnsGroup*>();
  e->dirty = true;
  if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming), "ens_create: event");
  if (!rc) rc = cuda_check(cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking), "ens_create: stream");
  if (!rc && precision == CHX_PREC_F32_REFINE) {
    e->sched = new (std::nothrow) EnsSchedule();
    if (!e->sched) rc = fail(CHX_ENOMEM, "ens_create: host allocation");
    if (!rc && (cudaMalloc(&e->sched->d_steps, kEnsMaxGroups * sizeof(FFStep)) != cudaSuccess ||
                cudaMalloc(&e->sched->d_order, kEnsMaxGroups * sizeof(int)) != cudaSuccess ||
                cudaMalloc(&e->sched->d_start, 3 * (kEnsMaxGroups + 1) * sizeof(int)) != cudaSuccess)) {
      cudaGetLastError();
      rc = fail(CHX_ENOMEM, "ens_create: schedule tables");
    }
  }
  if (rc) { ens_free(e); return rc; }
  *out = e;
  return CHX_OK;
}

extern "C" int ens_group_create(chx_ens* e, int n, double l, double gamma, int capacity, int* group_id) {
  if (!e || e->hdr.magic != kMagicEns || !group_id) return fail(CHX_EINVAL, "ens_group_create: bad argument");
  if (capacity < 1 || capacity > 65535) return fail(CHX_EINVAL, "ens_group_create: capacity %d", capacity);
  EnsGroup* G = new (std::nothrow) EnsGroup();
  if (!G) return fail(CHX_ENOMEM, "ens_group_create: host allocation");
  int rc = group_init(&G->g, n, n, l, l, gamma, e->dt, e->precision, capacity);
  if (rc) { free_group(G); return rc; }
  G->n = n; G->l = l; G->gamma = gamma; G->capacity = capacity;
  G->slot_gamma.assign(capacity, gamma);
  // room for the autotuner's larger segment counts (their boundary arrays grow with P)
  G->work_bytes = G->g.work_bytes + G->g.work_bytes / 4 + (1 << 20);
  G->bytes = state_bytes(n, capacity) + G->work_bytes + G->g.factor_bytes;
  if (e->budget && e->used + G->bytes > e->budget) {
    free_group(G);
    return fail(CHX_ENOMEM, "ens_group_create: %zu bytes over the HBM budget (%zu of %zu used)", G->bytes, e->used,
                e->budget);
  }
  const size_t sb = (size_t)capacity * n * n * sizeof(double);
  if (cudaMalloc(&G->d_state[0], sb) != cudaSuccess || cudaMalloc(&G->d_state[1], sb) != cudaSuccess ||
      cudaMalloc(&G->d_work, G->work_bytes) != cudaSuccess) {
    cudaGetLastError();
    free_group(G);
    return fail(CHX_ENOMEM, "ens_group_create: device allocation of %zu bytes", G->bytes);
  }
  if ((rc = cuda_check(cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking), "ens: stream")) ||
      (rc = cuda_check(cudaEventCreateWithFlags(&G->done, cudaEventDisableTiming), "ens: event"))) {
    free_group(G);
    return rc;
  }
  G->status = e->hdr.d_status;
  G->live = true;
  e->used += G->bytes;
  e->groups->push_back(G);
  *group_id = (int)e->groups->size() - 1;
  drop_graph(e);
  return CHX_OK;
}

extern "C" int ens_group_destroy(chx_ens* e, int group_id) {
  EnsGroup* G = get_group(e, group_id);
  if (!G) return fail(CHX_EINVAL, "ens_group_destroy: bad group %d", group_id);
  cudaDeviceSynchronize();
  e->used -= G->bytes;
  free_group(G);
  (*e->groups)[group_id] = nullptr;
  drop_graph(e);
  return CHX_OK;
}

extern "C" int ens_slot_load(chx_ens* e, int group_id, int slot, const double* c0, const double* cm1,
                             double gamma, void* stream) {
  EnsGroup* G = get_group(e, group_id);
  if (!G || !c0 || slot < 0 || slot >= G->capacity) return fail(CHX_EINVAL, "ens_slot_load: bad argument");
  const size_t nb = (size_t)G->n * G->n * sizeof(double);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = CHX_OK;
  if (gamma >= 0 && gamma != G->slot_gamma[slot]) {
    // the refactorisation uploads synchronously; wait for earlier work on the slot first
    rc = cuda_check(cudaStreamSynchronize(st), "ens_slot_load: synchronize");
    if (!rc) rc = group_set_gamma(&G->g, slot, gamma);
    if (rc) return rc;
    G->slot_gamma[slot] = gamma;
    drop_graph(e);  // the reduced-solve band and spike rows captured in the graph may have changed
  }
  rc = cuda_check(cudaMemcpyAsync((char*)G->d_state[G->cur] + slot * nb, c0, nb, cudaMemcpyDefault, st),
                      "ens_slot_load: C^n");
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync((char*)G->d_state[1 - G->cur] + slot * nb, cm1 ? cm1 : c0, nb, cudaMemcpyDefault,
                                    st),
                    "ens_slot_load: C^{n-1}");
  e->hdr.last_stream = st;
  return rc;
}

extern "C" int ens_slot_read(chx_ens* e, int group_id, int slot, double* c_now, double* c_prev, void* stream) {
  EnsGroup* G = get_group(e, group_id);
  if (!G || !c_now || slot < 0 || slot >= G->capacity) return fail(CHX_EINVAL, "ens_slot_read: bad argument");
  const size_t nb = (size_t)G->n * G->n * sizeof(double);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = cuda_check(cudaMemcpyAsync(c_now, (char*)G->d_state[G->cur] + slot * nb, nb, cudaMemcpyDefault, st),
                      "ens_slot_read");
  if (!rc && c_prev)
    rc = cuda_check(cudaMemcpyAsync(c_prev, (char*)G->d_state[1 - G->cur] + slot * nb, nb, cudaMemcpyDefault, st),
                    "ens_slot_read");
  e->hdr.last_stream = st;
  return rc;
}

extern "C" int ens_group_observables(chx_ens* e, int group_id, int with_k1, double* out, void* stream) {
  EnsGroup* G = get_group(e, group_id);
  if (!G || !out) return fail(CHX_EINVAL, "ens_group_observables: bad argument");
  if (G->active < 1) return CHX_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = group_observables(&G->g, G->active, G->d_state[G->cur], out, with_k1 ? 1 : 0, e->hdr.d_status, st);
  e->hdr.last_stream = st;
  return rc;
}

extern "C" int ens_slot_move(chx_ens* e, int group_id, int from, int to, void* stream) {
  EnsGroup* G = get_group(e, group_id);
  if (!G || from < 0 || to < 0 || from >= G->capacity || to >= G->capacity)
    return fail(CHX_EINVAL, "ens_slot_move: bad argument");
  if (from == to) return CHX_OK;
  const size_t nb = (size_t)G->n * G->n * sizeof(double);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = CHX_OK;
  for (int b = 0; b < 2 && !rc; ++b)
    rc = cuda_check(cudaMemcpyAsync((char*)G->d_state[b] + to * nb, (char*)G->d_state[b] + from * nb, nb,
                                    cudaMemcpyDeviceToDevice, st),
                    "ens_slot_move");
  if (!rc) rc = group_move_params(&G->g, from, to, st);
  if (!rc) G->slot_gamma[to] = G->slot_gamma[from];
  e->hdr.last_stream = st;
  return rc;
}

extern "C" int ens_group_set_cook(chx_ens* e, int group_id, double sigma, uint64_t seed, uint64_t step0) {
  EnsGroup* G = get_group(e, group_id);
  if (!G || !(sigma >= 0) || !isfinite(sigma)) return fail(CHX_EINVAL, "ens_group_set_cook: bad argument");
  int rc = cuda_check(cudaDeviceSynchronize(), "ens_group_set_cook: synchronize");
  if (rc) return rc;
  if (sigma == 0) {
    cudaFree(G->d_rho);
    cudaFree(G->d_step);
    G->d_rho = nullptr;
    G->d_step = nullptr;
    e->used -= G->cook_bytes;
    G->cook_bytes = 0;
    G->sigma = 0;
    G->g.noise = nullptr;
    drop_graph(e);
    return CHX_OK;
  }
  if (!G->d_rho) {
    const size_t bytes = 2 * (size_t)G->capacity * G->n * G->n * sizeof(double) + 256;
    if (e->budget && e->used + bytes > e->budget)
      return fail(CHX_ENOMEM, "ens_group_set_cook: %zu bytes of deviates over the HBM budget", bytes);
    if (cudaMalloc(&G->d_rho, bytes - 256) != cudaSuccess || cudaMalloc(&G->d_step, sizeof(uint64_t)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(G->d_rho);
      G->d_rho = nullptr;
      G->d_step = nullptr;
      return fail(CHX_ENOMEM, "ens_group_set_cook: device allocation of %zu bytes", bytes);
    }
    G->cook_bytes = bytes;
    e->used += bytes;
  }
  rc = cuda_check(cudaMemcpy(G->d_step, &step0, sizeof(uint64_t), cudaMemcpyHostToDevice), "ens_group_set_cook");
  if (rc) return rc;
  G->sigma = sigma;
  G->seed = seed;
  const double amp = sqrt(sigma / (G->g.dx * G->g.dy * G->g.dt));
  G->g.nkx = (2.0 / 3.0) * G->g.dt * amp / G->g.dx;
  G->g.nky = (2.0 / 3.0) * G->g.dt * amp / G->g.dy;
  drop_graph(e);
  return CHX_OK;
}

extern "C" int ens_group_set_active(chx_ens* e, int group_id, int active) {
  EnsGroup* G = get_group(e, group_id);
  if (!G || active < 0 || active > G->capacity) return fail(CHX_EINVAL, "ens_group_set_active: bad argument");
  if (G->active != active) {
    G->active = active;
    drop_graph(e);
  }
  return CHX_OK;
}

extern "C" int ens_step(chx_ens* e, int nsteps, void* stream) {
  if (!e || e->hdr.magic != kMagicEns || nsteps < 0) return fail(CHX_EINVAL, "ens_step: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = CHX_OK;
  if (nsteps >= 2 && (e->dirty || !e->exec)) {
    rc = build_graph(e);
    if (rc) return rc;
  }
  for (int k = 0; k + 2 <= nsteps; k += 2) {
    rc = cuda_check(cudaGraphLaunch(e->exec, st), "ens_step: graph launch");
    if (rc) return rc;
  }
  if (nsteps & 1) {
    if (packed(e) && !e->sched->valid) {
      rc = build_schedule(e);
      if (rc) return rc;
    }
    if (packed(e) && e->sched->valid) {
      step_packed(e, 0, st);
      for (EnsGroup* G : e->sched->members) G->cur = 1 - G->cur;
    } else {
      for (EnsGroup* G : *e->groups)
        if (G && G->live) step_group(G, st);
    }
    drop_graph(e);  // the captured pair and the schedule start from the other buffer now
  }
  e->hdr.last_stream = st;
  return launch_check("ens_step");
}

extern "C" int ens_group_step(chx_ens* e, int group_id, int nsteps, void* stream) {
  EnsGroup* G = get_group(e, group_id);
  if (!G || nsteps < 0) return fail(CHX_EINVAL, "ens_group_step: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  for (int k = 0; k < nsteps; ++k) step_group(G, st);
  if (nsteps & 1) drop_graph(e);
  e->hdr.last_stream = st;
  return launch_check("ens_group_step");
}

// Times `trial` steps of the group for each candidate pair of segment counts
// and keeps the fastest.  The state of the active slots is saved and restored
// around the trials, so the call changes no simulation.
// `trial` steps of group G's active slots with factors g by the packed phase
// launches the FP32 ensemble schedule runs, on a one-group schedule held in
// `dev` (room for one FFStep, then the order and the three phases' item
// ranges).  ms < 0: the candidate's tiles do not fit.  Steps G's state (the
// caller saves it) and flips G->cur per step.
static int time_packed_group(chx_ens* e, EnsGroup* G, ChGroup* g, int trial, void* dev, cudaStream_t st,
                             cudaEvent_t a, cudaEvent_t b, float* ms) {
  *ms = -1.f;
  FFStep P = ff_step_params(g, G->active, G->d_state[0], G->d_state[1], G->d_work, e->sched->target);
  P.cur0 = G->cur;
  if (P.xs < 1 || P.ysc < 1) return CHX_OK;
  const size_t smem[3] = {0, x_solve_smem(P.nx, P.ny, P.X.P, P.xs), y_solve_smem(P.ny, P.Y.P, P.ysc, P.yrb)};
  if (smem[1] > ens_phase_smem_max() || smem[2] > ens_phase_smem_max()) return CHX_OK;
  int items[3], host_ints[1 + 3 * 2], blocks[3], sms = 0, dv = 0;
  int rc = cuda_check(cudaGetDevice(&dv), "ens_autotune: device");
  if (!rc) rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dv), "ens_autotune: SMs");
  if (rc) return rc;
  host_ints[0] = 0;  // the order: the one group
  for (int ph = 0; ph < 3; ++ph) {
    items[ph] = ens_phase_items(ph, P);
    host_ints[1 + 2 * ph] = 0;
    host_ints[2 + 2 * ph] = items[ph];
    blocks[ph] = std::min(items[ph], sms * ens_phase_occupancy(ph, smem[ph]));
  }
  FFStep* d_steps = (FFStep*)dev;
  int* d_ints = (int*)((char*)dev + ((sizeof(FFStep) + 15) & ~(size_t)15));
  if ((rc = cuda_check(cudaMemcpy(d_steps, &P, sizeof(FFStep), cudaMemcpyHostToDevice), "ens_autotune: upload")) ||
      (rc = cuda_check(cudaMemcpy(d_ints, host_ints, sizeof(host_ints), cudaMemcpyHostToDevice), "ens_autotune: upload")))
    return rc;
  auto one = [&](int q) {
    for (int ph = 0; ph < 3; ++ph)
      launch_ens_phase_ff(ph, d_steps, d_ints, d_ints + 1 + 2 * ph, 1, items[ph], blocks[ph], q, smem[ph], st);
  };
  one(0);  // warm-up step
  cudaEventRecord(a, st);
  for (int k = 1; k <= trial; ++k) one(k & 1);
  cudaEventRecord(b, st);
  rc = cuda_check(cudaEventSynchronize(b), "ens_autotune: trial");
  if (!rc) cudaEventElapsedTime(ms, a, b);
  if ((1 + trial) & 1) G->cur = 1 - G->cur;
  return rc;
}

extern "C" int ens_autotune(chx_ens* e, int group_id, int trial, int* px_out, int* py_out, void* stream) {
  EnsGroup* G = get_group(e, group_id);
  if (!G || trial < 1) return fail(CHX_EINVAL, "ens_autotune: bad argument");
  if (G->active < 1) return fail(CHX_EINVAL, "ens_autotune: group %d has no active slots", group_id);
  cudaStream_t st = (cudaStream_t)stream;
  const int n = G->n;
  const size_t sb = (size_t)G->active * n * n * sizeof(double);
  std::vector<int> cx = segment_candidates(n, G->capacity * n, e->precision);
  double best = 1e300;
  int bx = G->g.X.P, by = G->g.Y.P;
  void* save = nullptr;
  if (e->budget && e->used + 2 * sb > e->budget)
    return fail(CHX_ENOMEM, "ens_autotune: %zu bytes of saved state over the HBM budget", 2 * sb);
  if (cudaMalloc(&save, 2 * sb) != cudaSuccess) {
    cudaGetLastError();
    return fail(CHX_ENOMEM, "ens_autotune: scratch for the saved state");
  }
  {
    cudaError_t ce = cudaMemcpyAsync(save, G->d_state[0], sb, cudaMemcpyDeviceToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync((char*)save + sb, G->d_state[1], sb, cudaMemcpyDeviceToDevice, st);
    if (ce != cudaSuccess) {
      cudaFree(save);
      return cuda_check(ce, "ens_autotune: saving the state");
    }
  }
  const int cur0 = G->cur;
  void* sched_scratch = nullptr;  // a one-group packed schedule (FP32 + refinement)
  if (packed(e) && cudaMalloc(&sched_scratch, 1024 + 64) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(save);
    return fail(CHX_ENOMEM, "ens_autotune: schedule scratch");
  }
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = cuda_check(cudaEventCreate(&a), "ens_autotune: event");
  if (!rc) rc = cuda_check(cudaEventCreate(&b), "ens_autotune: event");
  // one trial: `trial` steps of the group with px / py segments (ms, or < 0 when
  // the candidate does not fit the group's work buffer)
  auto trial_ms = [&](int px, int py, float* ms) -> int {
    *ms = -1.f;
    ChGroup trialg;
    int r = group_init(&trialg, n, n, G->l, G->l, G->gamma, e->dt, e->precision, G->capacity, px, py);
    if (r) return r;  // group_init frees its own partial allocations
    for (int z = 0; z < G->active && !r; ++z)
      if (G->slot_gamma[z] != G->gamma) r = group_set_gamma(&trialg, z, G->slot_gamma[z]);
    if (r || trialg.work_bytes > G->work_bytes) {  // a candidate that needs more scratch is skipped
      group_free(&trialg);
      return r;
    }
    if (packed(e)) {  // FP32 + refinement: timed as the ensemble runs it, by the packed phase launches
      r = time_packed_group(e, G, &trialg, trial, sched_scratch, st, a, b, ms);
      group_free(&trialg);
      return r;
    }
    group_step(&trialg, G->active, G->d_state[G->cur], G->d_state[1 - G->cur], G->d_work, 0, st, nullptr, G->status);
    G->cur = 1 - G->cur;
    cudaEventRecord(a, st);
    for (int k = 0; k < trial; ++k) {
      group_step(&trialg, G->active, G->d_state[G->cur], G->d_state[1 - G->cur], G->d_work, 0, st, nullptr, G->status);
      G->cur = 1 - G->cur;
    }
    cudaEventRecord(b, st);
    r = cuda_check(cudaEventSynchronize(b), "ens_autotune: trial");
    if (!r) cudaEventElapsedTime(ms, a, b);
    group_free(&trialg);
    return r;
  };
  // coordinate search: the x count with y's fixed, then the y count with x's chosen
  for (int pass = 0; pass < 2 && !rc; ++pass) {
    for (int P : cx) {
      const int px = pass == 0 ? P : bx, py = pass == 0 ? by : P;
      float ms = -1.f;
      rc = trial_ms(px, py, &ms);
      if (rc) break;
      if (ms >= 0.f && ms < best) {
        best = ms;
        bx = px;
        by = py;
      }
    }
  }
  // put the state back (whatever the trials returned)
  int rs = cuda_check(cudaMemcpyAsync(G->d_state[0], save, sb, cudaMemcpyDeviceToDevice, st), "ens_autotune: restore");
  if (!rs) rs = cuda_check(cudaMemcpyAsync(G->d_state[1], (char*)save + sb, sb, cudaMemcpyDeviceToDevice, st),
                           "ens_autotune: restore");
  if (!rs) rs = cuda_check(cudaStreamSynchronize(st), "ens_autotune: restore");
  if (!rc) rc = rs;
  G->cur = cur0;
  cudaFree(save);
  cudaFree(sched_scratch);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (rc) return rc;
  if (bx != G->g.X.P || by != G->g.Y.P) {
    ChGroup ng;
    rc = group_init(&ng, n, n, G->l, G->l, G->gamma, e->dt, e->precision, G->capacity, bx, by);
    for (int z = 0; z < G->capacity && !rc; ++z)
      if (G->slot_gamma[z] != G->gamma) rc = group_set_gamma(&ng, z, G->slot_gamma[z]);
    // the new segment counts change the factor arrays' size
    const size_t nbytes = state_bytes(n, G->capacity) + G->work_bytes + ng.factor_bytes;
    if (!rc && e->budget && e->used - G->bytes + nbytes > e->budget)
      rc = fail(CHX_ENOMEM, "ens_autotune: factors for %d x %d segments over the HBM budget", bx, by);
    if (rc) {
      group_free(&ng);
      return rc;
    }
    const double nkx = G->g.nkx, nky = G->g.nky;
    group_free(&G->g);
    G->g = ng;
    e->used = e->used - G->bytes + nbytes;
    G->bytes = nbytes;
    G->g.nkx = nkx;  // the group's forcing weights carry over to the new factors
    G->g.nky = nky;
    drop_graph(e);
  }
  if (px_out) *px_out = G->g.X.P;
  if (py_out) *py_out = G->g.Y.P;
  return CHX_OK;
}

extern "C" int ens_info(chx_ens* e, int group_id, int* n, int* capacity, int* active, int* px, int* py,
                        size_t* bytes) {
  EnsGroup* G = get_group(e, group_id);
  if (!G) return fail(CHX_EINVAL, "ens_info: bad group %d", group_id);
  if (n) *n = G->n;
  if (capacity) *capacity = G->capacity;
  if (active) *active = G->active;
  if (px) *px = G->g.X.P;
  if (py) *py = G->g.Y.P;
  if (bytes) *bytes = G->bytes;
  return CHX_OK;
}

extern "C" size_t ens_bytes_used(const chx_ens* e) { return (e && e->hdr.magic == kMagicEns) ? e->used : 0; }

// Times `trial` packed steps for each candidate schedule of an FP32 +
// refinement ensemble and keeps the fastest: the group order (most or least
// work per item first), the points per work item of the solves (2048, 4096 or
// 8192: every group's x rows and y columns per block follow from it) and the y
// phase's blocks per SM (as many as fit, or one).  The trials overwrite
// C^{n-1} of the active slots, which is saved first and put back, so the call
// changes no simulation; the save counts against the HBM budget.
extern "C" int ens_tune_schedule(chx_ens* e, int trial, int* order_out, int* target_out, int* blocks_out,
                                 void* stream) {
  if (!e || e->hdr.magic != kMagicEns || trial < 1) return fail(CHX_EINVAL, "ens_tune_schedule: bad argument");
  if (!packed(e)) return fail(CHX_EUNSUPPORTED, "ens_tune_schedule: FP32 + refinement ensembles only");
  cudaStream_t st = (cudaStream_t)stream;
  EnsSchedule& S = *e->sched;
  int rc = build_schedule(e);
  if (rc) return rc;
  if (!S.valid) return fail(CHX_EUNSUPPORTED, "ens_tune_schedule: no active groups, or more than %d", kEnsMaxGroups);
  // save C^{n-1} of every active slot
  size_t save_bytes = 0;
  for (EnsGroup* G : S.members) save_bytes += (size_t)G->active * G->n * G->n * sizeof(double);
  if (e->budget && e->used + save_bytes > e->budget)
    return fail(CHX_ENOMEM, "ens_tune_schedule: %zu bytes of saved state over the HBM budget", save_bytes);
  char* save = nullptr;
  if (cudaMalloc(&save, save_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(CHX_ENOMEM, "ens_tune_schedule: %zu bytes for the saved state", save_bytes);
  }
  {
    size_t off = 0;
    for (EnsGroup* G : S.members) {
      const size_t b = (size_t)G->active * G->n * G->n * sizeof(double);
      const cudaError_t ce = cudaMemcpyAsync(save + off, G->d_state[1 - G->cur], b, cudaMemcpyDeviceToDevice, st);
      if (ce != cudaSuccess) {
        cudaFree(save);
        return cuda_check(ce, "ens_tune_schedule: saving the state");
      }
      off += b;
    }
  }
  cudaEvent_t a = nullptr, b = nullptr;
  rc = cuda_check(cudaEventCreate(&a), "ens_tune_schedule: event");
  if (!rc) rc = cuda_check(cudaEventCreate(&b), "ens_tune_schedule: event");
  const int order0 = S.order_mode, target0 = S.target, bps0 = S.bps[2];
  double best = 1e300;
  int bo = order0, bt = target0, bb = bps0;
  for (int om = 0; om < 2 && !rc; ++om)
    for (int tg : {2048, 4096, 8192}) {
      if (rc) break;
      for (int yb : {0, 1}) {
        S.order_mode = om;
        S.target = tg;
        S.bps[2] = yb;
        if ((rc = build_schedule(e))) break;
        if (!S.valid) continue;
        step_packed(e, 0, st);  // warm-up
        cudaEventRecord(a, st);
        for (int k = 0; k < trial; ++k) step_packed(e, 0, st);
        cudaEventRecord(b, st);
        if ((rc = cuda_check(cudaEventSynchronize(b), "ens_tune_schedule: trial"))) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) {
          best = ms;
          bo = om;
          bt = tg;
          bb = yb;
        }
      }
    }
  {
    // put C^{n-1} back (whatever the trials returned)
    size_t off = 0;
    int rs = CHX_OK;
    for (EnsGroup* G : S.members) {
      const size_t bs = (size_t)G->active * G->n * G->n * sizeof(double);
      if (!rs)
        rs = cuda_check(cudaMemcpyAsync(G->d_state[1 - G->cur], save + off, bs, cudaMemcpyDeviceToDevice, st),
                        "ens_tune_schedule: restore");
      off += bs;
    }
    if (!rs) rs = cuda_check(cudaStreamSynchronize(st), "ens_tune_schedule: restore");
    if (!rc) rc = rs;
  }
  cudaFree(save);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  S.order_mode = rc ? order0 : bo;
  S.target = rc ? target0 : bt;
  S.bps[2] = rc ? bps0 : bb;
  drop_graph(e);
  if (rc) return rc;
  rc = build_schedule(e);
  if (rc) return rc;
  if (order_out) *order_out = S.order_mode;
  if (target_out) *target_out = S.target;
  if (blocks_out)
    for (int ph = 0; ph < 3; ++ph) blocks_out[ph] = S.blocks[ph];
  return CHX_OK;
}

// The packed schedule's layout for the current groups (FP32 + refinement
// ensembles): work items and blocks of each phase, points per item, order.
extern "C" int ens_schedule_info(chx_ens* e, int* items_out, int* blocks_out, int* target_out, int* order_out) {
  if (!e || e->hdr.magic != kMagicEns) return fail(CHX_EINVAL, "ens_schedule_info: bad argument");
  if (!packed(e)) return fail(CHX_EUNSUPPORTED, "ens_schedule_info: FP32 + refinement ensembles only");
  EnsSchedule& S = *e->sched;
  if (!S.valid) {
    int rc = build_schedule(e);
    if (rc) return rc;
  }
  for (int ph = 0; ph < 3; ++ph) {
    if (items_out) items_out[ph] = S.valid ? S.nitems[ph] : 0;
    if (blocks_out) blocks_out[ph] = S.valid ? S.blocks[ph] : 0;
  }
  if (target_out) *target_out = S.target;
  if (order_out) *order_out = S.order_mode;
  return CHX_OK;
}
