// Batched execution of many solves: the runtime behind lbm_batch_* (include/lbm_mrt.h).
//
// Members are grouped by (lattice object, storage dtype, equation, per-order rates or not). Each
// group gets its lattice
// tables (kernel parameter), one descriptor per solve and a tile work-list covering every cell of
// every solve; one persistent launch per group advances all its solves by one time step. The
// launches of CHUNK consecutive steps are captured once in a CUDA graph and replayed; membership or
// parameter changes mark the batch dirty and the next step rebuilds groups and graph.
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "lbm_internal.cuh"

namespace {

constexpr int kChunk = 8;  // steps per captured graph (even: each model's buffers return to place)

struct GroupHost {
  lbm::BatchGroup g;
  lbm::BatchTables<float> tables;
  std::vector<lbm::SolveDesc<float>> desc;
  std::vector<lbm::HighParams<float>> high;  // per solve, for a group with per-order rates
  std::vector<lbm_model*> members;
};

}  // namespace

struct DeviceBuffers {
  void* desc = nullptr;
  size_t desc_cap = 0;
  void* tiles = nullptr;
  size_t tiles_cap = 0;
  void* high = nullptr;
  size_t high_cap = 0;
};

struct lbm_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  int max_solves = 0;
  int num_sms = 0;
  std::vector<lbm_model*> members;
  std::vector<GroupHost> groups;
  // members of at least solo_cells cells run on the single-solve kernels (one launch per step
  // each, outside the work-lists): large grids fill the GPU alone and the single-solve kernels
  // reach a larger share of HBM bandwidth than the work-list kernel
  std::vector<lbm_model*> solos;
  int64_t solo_cells = int64_t(1) << 19;
  // the solos' launches run on a second stream, forked from the batch stream before the
  // work-list launches of a step call and joined back after them, so that a large solve's
  // bandwidth-bound steps and the small solves' latency-bound ones share the SMs
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  // one stream per group: a step call forks them from the batch stream, each runs its group's
  // steps as a chain, and the batch stream joins them all, so that groups too small to fill the
  // GPU (the 2D solves of a serving mix) overlap instead of queueing one launch after another.
  // The events of a graph capture are separate from those of the launches outside one.
  std::vector<cudaStream_t> lanes;
  std::vector<cudaEvent_t> lane_join, cap_join;
  cudaEvent_t lane_fork = nullptr, cap_fork = nullptr;
  std::map<std::tuple<int, int, int>, int> tile;  // (kind, store, eq) -> cells per tile
  std::map<std::tuple<int, int, int>, int> per_sm;  // (kind, store, eq) -> resident blocks per SM (cap)
  bool dirty = true;
  bool stable = false;  // no change since the last step call: capture a graph
  cudaGraphExec_t graph = nullptr;
  // replaced graphs whose launches may still run, each with an event recorded after them on the
  // batch stream: destroyed once the event has completed (no host synchronisation)
  std::vector<std::pair<cudaGraphExec_t, cudaEvent_t>> old_graphs;
  // work-list buffers by group key, kept across rebuilds and grown geometrically
  std::map<std::tuple<const lbm_lattice*, int, int, int>, DeviceBuffers> buffers;
  int64_t steps = 0, launches = 0, rebuilds = 0, captures = 0;
};

namespace lbm {

void batch_mark_dirty(lbm_batch* b) {
  if (b) b->dirty = true;
}

namespace {

template <class F>
lbm_status dispatch_batch_kind(int kind, F&& f) {
  switch (kind) {
    case LBM_RD2Q13: return f(std::integral_constant<int, LBM_RD2Q13>{});
    case LBM_RD2Q17: return f(std::integral_constant<int, LBM_RD2Q17>{});
    case LBM_RD2Q21: return f(std::integral_constant<int, LBM_RD2Q21>{});
    case LBM_RD2Q25: return f(std::integral_constant<int, LBM_RD2Q25>{});
    case LBM_RD3Q33: return f(std::integral_constant<int, LBM_RD3Q33>{});
    case LBM_RD3Q45: return f(std::integral_constant<int, LBM_RD3Q45>{});
    case LBM_RD3Q53: return f(std::integral_constant<int, LBM_RD3Q53>{});
    case LBM_RD2Q9: return f(std::integral_constant<int, LBM_RD2Q9>{});
    case LBM_RD3Q27: return f(std::integral_constant<int, LBM_RD3Q27>{});
  }
  return set_error(LBM_ERR_ARG, "unknown lattice kind");
}

// Destroy the replaced graphs whose launches have completed (all of them when `all`, after the
// caller has synchronised the batch stream).
void reap_graphs(lbm_batch* b, bool all) {
  std::vector<std::pair<cudaGraphExec_t, cudaEvent_t>> keep;
  for (auto& ge : b->old_graphs) {
    if (all || cudaEventQuery(ge.second) == cudaSuccess) {
      cudaGraphExecDestroy(ge.first);
      cudaEventDestroy(ge.second);
    } else {
      keep.push_back(ge);
    }
  }
  cudaGetLastError();  // clear the not-ready status of the queries
  b->old_graphs.swap(keep);
}

void drop_graph(lbm_batch* b) {
  reap_graphs(b, false);
  if (b->graph) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventRecord(ev, b->stream) == cudaSuccess) {
      b->old_graphs.emplace_back(b->graph, ev);
    } else {  // no event: wait for the launches before destroying the graph
      if (ev) cudaEventDestroy(ev);
      cudaStreamSynchronize(b->stream);
      cudaGraphExecDestroy(b->graph);
    }
    b->graph = nullptr;
  }
}

void free_groups(lbm_batch* b) {
  b->groups.clear();
  drop_graph(b);
}

void free_buffers(lbm_batch* b) {
  for (auto& kv : b->buffers) {
    if (kv.second.desc) cudaFree(kv.second.desc);
    if (kv.second.tiles) cudaFree(kv.second.tiles);
    if (kv.second.high) cudaFree(kv.second.high);
  }
  b->buffers.clear();
}

cudaError_t ensure(void** ptr, size_t* cap, size_t bytes) {
  if (bytes <= *cap) return cudaSuccess;
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  size_t want = std::max(bytes, *cap * 2);
  cudaError_t err = cudaMalloc(ptr, want);
  *cap = err == cudaSuccess ? want : 0;
  return err;
}

void fill_desc(const lbm_model* m, SolveDesc<float>* d) {
  StepParams<float> p;
  make_step_params<float>(m, &p);
  std::memset(d, 0, sizeof(*d));
  for (int r = 0; r < kMaxR; ++r) {
    d->sd[r] = p.sd[r];
    d->half[r] = p.half[r];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      d->sdn[i][j] = p.sdn[i][j];
      d->halfn[i][j] = p.halfn[i][j];
    }
  d->s_high = p.s_high;
  d->one_minus_sh = p.one_minus_sh;
  d->sh_rho_ref = p.sh_rho_ref;
  d->cs2_eq = p.cs2_eq;
  d->nonlin_third = p.nonlin_third;
  for (int a = 0; a < 3; ++a) {
    d->u_const[a] = p.u_const[a];
    d->n[a] = p.n[a];
  }
  d->ncells = p.ncells;
  for (int a = 0; a < 2; ++a) {
    d->div_m[a] = p.div_m[a];
    d->div_s[a] = p.div_s[a];
  }
  d->force_a = p.force_a;
  d->force_b = p.force_b;
  d->force_tab = p.force_tab;
  d->f[0] = m->f[m->cur];
  d->f[1] = m->f[m->cur ^ 1];
  d->phi = static_cast<float*>(m->phi_prev);
  d->ncde_variant = p.ncde_variant;
  for (int a = 0; a < 3; ++a) {
    d->kfac[a] = p.kfac[a];
    d->cde_coef[a] = p.cde_coef[a];
    d->gscale[a] = p.gscale[a];
  }
  d->nonlin_rate = p.nonlin_rate;
  d->a1 = p.a1;
  d->half0 = p.half0;
  d->grad_on = p.grad_on;
  if (m->eq == LBM_NSE && m->m2g_aniso) {
    // the density history ping-pongs with the populations: parity k reads hist[k], writes hist[k ^ 1]
    d->grad_in[0] = static_cast<const float*>(m->rho_hist[m->hist_cur]);
    d->grad_in[1] = static_cast<const float*>(m->rho_hist[m->hist_cur ^ 1]);
    d->rho_out[0] = static_cast<float*>(m->rho_hist[m->hist_cur ^ 1]);
    d->rho_out[1] = static_cast<float*>(m->rho_hist[m->hist_cur]);
  } else if (p.grad_on) {
    d->grad_in[0] = d->grad_in[1] = p.grad_in;   // the cross-diffusion field psi
  }
}

lbm_status launch_group(const GroupHost& gh, int parity, cudaStream_t stream) {
  return dispatch_batch_kind(gh.g.kind, [&](auto kc) {
    return BatchLaunch<decltype(kc)::value>::launch(gh.g, parity, stream);
  });
}

// streams and events for the group lanes (created once, grown with the group count)
lbm_status ensure_lanes(lbm_batch* b) {
  cudaError_t err = cudaSuccess;
  if (!b->lane_fork) err = cudaEventCreateWithFlags(&b->lane_fork, cudaEventDisableTiming);
  if (err == cudaSuccess && !b->cap_fork) err = cudaEventCreateWithFlags(&b->cap_fork, cudaEventDisableTiming);
  while (err == cudaSuccess && b->lanes.size() < b->groups.size()) {
    cudaStream_t st = nullptr;
    cudaEvent_t e1 = nullptr, e2 = nullptr;
    err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e1, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e2, cudaEventDisableTiming);
    if (err != cudaSuccess) {
      if (st) cudaStreamDestroy(st);
      if (e1) cudaEventDestroy(e1);
      break;
    }
    b->lanes.push_back(st);
    b->lane_join.push_back(e1);
    b->cap_join.push_back(e2);
  }
  return err == cudaSuccess ? LBM_OK : cuda_error(err, "batch group streams");
}

// nsteps steps of every group, as one chain per group on its lane: forked from `main` and joined
// back into it (inside a graph capture of `main` too, with the capture's own events). Step s of
// the call reads the buffers of parity s & 1. One group runs on `main` itself.
lbm_status launch_groups(lbm_batch* b, int nsteps, cudaStream_t main, bool capturing) {
  if (b->groups.size() == 1) {
    for (int s = 0; s < nsteps; ++s) {
      lbm_status st = launch_group(b->groups[0], s & 1, main);
      if (st != LBM_OK) return st;
    }
    return LBM_OK;
  }
  lbm_status st = ensure_lanes(b);
  if (st != LBM_OK) return st;
  cudaEvent_t fork = capturing ? b->cap_fork : b->lane_fork;
  cudaError_t err = cudaEventRecord(fork, main);
  if (err != cudaSuccess) return cuda_error(err, "batch group fork");
  for (size_t k = 0; k < b->groups.size(); ++k) {
    cudaStream_t lane = b->lanes[k];
    err = cudaStreamWaitEvent(lane, fork, 0);
    if (err != cudaSuccess) return cuda_error(err, "batch group fork");
    for (int s = 0; s < nsteps && st == LBM_OK; ++s) st = launch_group(b->groups[k], s & 1, lane);
    // joined even after a failed launch, so that nothing on the lane is left outside the batch stream
    cudaEvent_t done = capturing ? b->cap_join[k] : b->lane_join[k];
    err = cudaEventRecord(done, lane);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(main, done, 0);
    if (err != cudaSuccess) return cuda_error(err, "batch group join");
    if (st != LBM_OK) return st;
  }
  return LBM_OK;
}

lbm_status upload_desc(lbm_batch* b, GroupHost& gh) {
  cudaError_t err = cudaMemcpyAsync(gh.g.d_desc, gh.desc.data(), gh.desc.size() * sizeof(SolveDesc<float>),
                                    cudaMemcpyHostToDevice, b->stream);
  return err == cudaSuccess ? LBM_OK : cuda_error(err, "batch descriptor upload");
}

lbm_status rebuild(lbm_batch* b) {
  free_groups(b);
  b->solos.clear();
  std::map<std::tuple<const lbm_lattice*, int, int, int>, size_t> index;
  for (lbm_model* m : b->members) {
    if (b->solo_cells > 0 && m->ncells >= b->solo_cells) {
      b->solos.push_back(m);
      continue;
    }
    const int high = has_high_rates(m) ? 1 : 0;
    auto key = std::make_tuple(m->lat, m->store, m->eq, high);
    auto it = index.find(key);
    if (it == index.end()) {
      index[key] = b->groups.size();
      b->groups.emplace_back();
      GroupHost& gh = b->groups.back();
      std::memset(&gh.g, 0, sizeof(gh.g));
      gh.g.kind = m->lat->kind;
      gh.g.store = m->store;
      gh.g.eq = m->eq;
      gh.g.lat = m->lat;
      gh.g.high = high;
      auto t = b->tile.find(std::make_tuple(m->lat->kind, m->store, m->eq));
      gh.g.block = high || t == b->tile.end() ? kBlock : t->second;
      StepParams<float> p;
      make_step_params<float>(m, &p);
      std::memcpy(gh.tables.T, p.T, sizeof(p.T));
      std::memcpy(gh.tables.D, p.D, sizeof(p.D));
      std::memcpy(gh.tables.invN, p.invN, sizeof(p.invN));
      std::memcpy(gh.tables.w, p.w, sizeof(p.w));
      std::memcpy(gh.tables.wref, p.wref, sizeof(p.wref));
      std::memcpy(gh.tables.wmom_ref, p.wmom_ref, sizeof(p.wmom_ref));
      gh.members.push_back(m);
    } else {
      b->groups[it->second].members.push_back(m);
    }
  }
  for (auto& gh : b->groups) {
    gh.g.tables = &gh.tables;
    gh.desc.resize(gh.members.size());
    gh.high.resize(gh.g.high ? gh.members.size() : 0);
    std::vector<Tile> tiles;
    for (size_t j = 0; j < gh.members.size(); ++j) {
      fill_desc(gh.members[j], &gh.desc[j]);
      if (gh.g.high) make_high_params<float>(gh.members[j], &gh.high[j]);
      for (int c0 = 0; c0 < gh.members[j]->ncells; c0 += gh.g.block) tiles.push_back(Tile{int(j), c0});
    }
    gh.g.nsolves = int(gh.members.size());
    gh.g.ntiles = int(tiles.size());
    // The previous work-list may still be read by launches queued on the batch stream: the new one
    // is uploaded on that stream, so it lands after them (a buffer that must grow is freed by
    // cudaFree, which waits for the device); the host vectors are staged by the copy call itself.
    DeviceBuffers& buf = b->buffers[std::make_tuple(gh.g.lat, gh.g.store, gh.g.eq, gh.g.high)];
    cudaError_t err = ensure(&buf.desc, &buf.desc_cap, gh.desc.size() * sizeof(SolveDesc<float>));
    if (err == cudaSuccess) err = ensure(&buf.tiles, &buf.tiles_cap, tiles.size() * sizeof(Tile));
    if (err == cudaSuccess && gh.g.high)
      err = ensure(&buf.high, &buf.high_cap, gh.high.size() * sizeof(HighParams<float>));
    gh.g.d_desc = buf.desc;
    gh.g.d_tiles = static_cast<Tile*>(buf.tiles);
    gh.g.d_high = gh.g.high ? buf.high : nullptr;
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(gh.g.d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice,
                            b->stream);
    if (err == cudaSuccess && gh.g.high)
      err = cudaMemcpyAsync(gh.g.d_high, gh.high.data(), gh.high.size() * sizeof(HighParams<float>),
                            cudaMemcpyHostToDevice, b->stream);
    if (err != cudaSuccess) return cuda_error(err, "batch work-list allocation");
    lbm_status st = upload_desc(b, gh);
    if (st != LBM_OK) return st;
    int per_sm = 0;
    st = dispatch_batch_kind(gh.g.kind, [&](auto kc) {
      return BatchLaunch<decltype(kc)::value>::occupancy(gh.g.store, gh.g.eq, gh.g.block, gh.g.high, &per_sm);
    });
    if (st != LBM_OK) return st;
    auto cap = b->per_sm.find(std::make_tuple(gh.g.kind, gh.g.store, gh.g.eq));
    if (cap != b->per_sm.end() && cap->second > 0) per_sm = std::min(std::max(1, per_sm), cap->second);
    gh.g.grid = std::max(1, std::min(gh.g.ntiles, std::max(1, per_sm) * b->num_sms));
  }
  b->dirty = false;
  b->stable = false;
  b->rebuilds += 1;
  return LBM_OK;
}

lbm_status capture(lbm_batch* b) {
  drop_graph(b);
  if (!b->groups.empty()) {
    if (b->groups.size() > 1) {  // streams and events are created before the capture begins
      lbm_status st = ensure_lanes(b);
      if (st != LBM_OK) return st;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t err = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return cuda_error(err, "graph capture (the batch needs a non-legacy stream)");
    const lbm_status st = launch_groups(b, kChunk, b->stream, true);
    err = cudaStreamEndCapture(b->stream, &graph);
    if (st != LBM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (err != cudaSuccess) return cuda_error(err, "graph capture");
    err = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) return cuda_error(err, "graph instantiation");
  }
  b->captures += 1;
  return LBM_OK;
}

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceScope() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

lbm_status lbm_batch_create(void* stream, int max_solves, lbm_batch** out) {
  if (!out) return set_error(LBM_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (max_solves < 1) return set_error(LBM_ERR_ARG, "max_solves must be positive");
  auto* b = new (std::nothrow) lbm_batch;
  if (!b) return set_error(LBM_ERR_OOM, "host allocation failed");
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  b->max_solves = max_solves;
  if (stream) {
    b->stream = static_cast<cudaStream_t>(stream);
  } else {
    cudaError_t err = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (err != cudaSuccess) {
      delete b;
      return cuda_error(err, "batch stream");
    }
    b->owns_stream = true;
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_add(lbm_batch* b, lbm_model* m) {
  if (!b || !m) return set_error(LBM_ERR_ARG, "NULL argument");
  if (m->batch) return set_error(LBM_ERR_ARG, "model is already in a batch");
  if (m->device != b->device) return set_error(LBM_ERR_ARG, "model and batch are on different devices");
  if (m->store == LBM_F64) return set_error(LBM_ERR_NOT_IMPLEMENTED, "batched execution supports F32 and 16-bit storage");
  if (int(b->members.size()) >= b->max_solves) return set_error(LBM_ERR_ARG, "batch is full");
  DeviceScope scope(b->device);
  cudaError_t err = cudaStreamSynchronize(m->stream);
  if (err != cudaSuccess) return cuda_error(err, "model stream");
  m->own_stream = m->stream;
  m->stream = b->stream;
  m->batch = b;
  b->members.push_back(m);
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_remove(lbm_batch* b, lbm_model* m) {
  if (!b || !m) return set_error(LBM_ERR_ARG, "NULL argument");
  auto it = std::find(b->members.begin(), b->members.end(), m);
  if (it == b->members.end() || m->batch != b) return set_error(LBM_ERR_ARG, "model is not in this batch");
  DeviceScope scope(b->device);
  // hand the model back to its own stream after the batch's queued steps, without waiting on the
  // host: the model's stream waits for an event recorded on the batch stream
  cudaEvent_t ev = nullptr;
  cudaError_t err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (err == cudaSuccess) err = cudaEventRecord(ev, b->stream);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(m->own_stream, ev, 0);
  if (ev) cudaEventDestroy(ev);
  if (err != cudaSuccess) return cuda_error(err, "batch stream hand-over");
  b->members.erase(it);
  m->stream = m->own_stream;
  m->batch = nullptr;
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_set_tile(lbm_batch* b, lbm_kind kind, lbm_dtype store, lbm_eq eq, int cells_per_tile) {
  if (!b) return set_error(LBM_ERR_ARG, "NULL batch");
  if (cells_per_tile != 64 && cells_per_tile != 128 && cells_per_tile != 256)
    return set_error(LBM_ERR_ARG, "cells per tile must be 64, 128 or 256");
  b->tile[std::make_tuple(int(kind), int(store), int(eq))] = cells_per_tile;
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_set_blocks_per_sm(lbm_batch* b, lbm_kind kind, lbm_dtype store, lbm_eq eq, int blocks) {
  if (!b) return set_error(LBM_ERR_ARG, "NULL batch");
  if (blocks < 0) return set_error(LBM_ERR_ARG, "blocks per SM must be non-negative");
  b->per_sm[std::make_tuple(int(kind), int(store), int(eq))] = blocks;
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_set_solo_threshold(lbm_batch* b, int64_t cells) {
  if (!b) return set_error(LBM_ERR_ARG, "NULL batch");
  if (cells < 0) return set_error(LBM_ERR_ARG, "the threshold must be non-negative");
  b->solo_cells = cells;
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps) {
  if (!b) return set_error(LBM_ERR_ARG, "NULL batch");
  if (nsteps < 0) return set_error(LBM_ERR_ARG, "nsteps must be non-negative");
  if (b->members.empty() || nsteps == 0) return LBM_OK;
  DeviceScope scope(b->device);
  if (b->dirty) {
    lbm_status st = rebuild(b);
    if (st != LBM_OK) return st;
  } else if (b->stable && !b->graph && nsteps >= kChunk) {
    // membership unchanged over a whole call: capture the steps in a graph from now on
    lbm_status st = capture(b);
    if (st != LBM_OK) return st;
  }
  const bool use_graph = b->graph != nullptr;
  const int64_t chunks = use_graph ? nsteps / kChunk : 0;
  const int rem = int(nsteps - chunks * kChunk);
  // the solos first, on the side stream (ordered after everything queued on the batch stream)
  const bool forked = !b->solos.empty();
  if (forked) {
    cudaError_t err = cudaSuccess;
    if (!b->side) err = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (err == cudaSuccess && !b->fork) err = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (err == cudaSuccess && !b->join) err = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventRecord(b->fork, b->stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(b->side, b->fork, 0);
    if (err != cudaSuccess) return cuda_error(err, "batch side stream");
  }
  lbm_status st = LBM_OK;
  for (lbm_model* m : b->solos) {
    const cudaStream_t own = m->stream;  // the batch stream while the model is a member
    m->stream = b->side;
    st = dispatch_batch_kind(m->lat->kind, [&](auto kc) {
      return Launch<decltype(kc)::value>::step(m, nsteps, true);
    });
    m->stream = own;
    if (st != LBM_OK) break;
  }
  for (int64_t c = 0; c < chunks && st == LBM_OK; ++c) {
    cudaError_t err = cudaGraphLaunch(b->graph, b->stream);
    if (err != cudaSuccess) st = cuda_error(err, "batch graph launch");
  }
  if (rem > 0 && st == LBM_OK && !b->groups.empty()) st = launch_groups(b, rem, b->stream, false);
  if (forked) {  // join, also after a failed launch: nothing queued on the side stream is left behind
    cudaError_t err = cudaEventRecord(b->join, b->side);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(b->stream, b->join, 0);
    if (err != cudaSuccess && st == LBM_OK) st = cuda_error(err, "batch side stream");
  }
  if (st != LBM_OK) return st;
  if (rem & 1) {
    // every model's current buffer flipped: swap the descriptors' buffers (the graph reads them)
    for (auto& gh : b->groups) {
      for (size_t j = 0; j < gh.members.size(); ++j) {
        lbm_model* m = gh.members[j];
        m->cur ^= 1;
        std::swap(gh.desc[j].f[0], gh.desc[j].f[1]);
        if (m->eq == LBM_NSE && m->m2g_aniso) {
          m->hist_cur ^= 1;
          std::swap(gh.desc[j].grad_in[0], gh.desc[j].grad_in[1]);
          std::swap(gh.desc[j].rho_out[0], gh.desc[j].rho_out[1]);
        }
      }
      const lbm_status su = upload_desc(b, gh);
      if (su != LBM_OK) return su;
    }
  }
  for (auto& gh : b->groups)  // (the single-solve launcher counts the solos' steps itself)
    for (lbm_model* m : gh.members) {
      m->steps += nsteps;
      m->launches += nsteps;
    }
  b->steps += nsteps;
  b->launches += nsteps * int64_t(b->groups.size() + b->solos.size());
  b->stable = true;
  return LBM_OK;
}

lbm_status lbm_batch_counters(const lbm_batch* b, int64_t* steps, int64_t* launches, int* groups, int64_t* tiles) {
  if (!b) return set_error(LBM_ERR_ARG, "NULL batch");
  if (steps) *steps = b->steps;
  if (launches) *launches = b->launches;
  if (groups) *groups = int(b->groups.size());
  if (tiles) {
    int64_t t = 0;
    for (const auto& gh : b->groups) t += gh.g.ntiles;
    *tiles = t;
  }
  return LBM_OK;
}

lbm_status lbm_batch_synchronize(lbm_batch* b) {
  if (!b) return set_error(LBM_ERR_ARG, "NULL batch");
  DeviceScope scope(b->device);
  cudaError_t err = cudaStreamSynchronize(b->stream);
  return err == cudaSuccess ? LBM_OK : cuda_error(err, "batch synchronize");
}

void* lbm_batch_stream(const lbm_batch* b) { return b ? static_cast<void*>(b->stream) : nullptr; }

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  DeviceScope scope(b->device);
  cudaStreamSynchronize(b->stream);
  for (lbm_model* m : b->members) {
    m->stream = m->own_stream;
    m->batch = nullptr;
  }
  if (b->side) cudaStreamSynchronize(b->side);
  for (cudaStream_t lane : b->lanes) cudaStreamSynchronize(lane);
  free_groups(b);
  reap_graphs(b, true);
  free_buffers(b);
  for (size_t k = 0; k < b->lanes.size(); ++k) {
    cudaStreamDestroy(b->lanes[k]);
    cudaEventDestroy(b->lane_join[k]);
    cudaEventDestroy(b->cap_join[k]);
  }
  if (b->lane_fork) cudaEventDestroy(b->lane_fork);
  if (b->cap_fork) cudaEventDestroy(b->cap_fork);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->owns_stream) cudaStreamDestroy(b->stream);
  delete b;
  return LBM_OK;
}

}  // extern "C"
