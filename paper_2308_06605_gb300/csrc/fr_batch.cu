// Batched RK stages for ensembles of independent meshes (include/fr.h, fr_batch_*): every stage
// of every case in one cooperative persistent launch, captured in a CUDA graph per stage.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fr_device.hpp"

using namespace frx;

struct fr_batch {
  std::vector<fr_mesh *> meshes;
  std::vector<BatchCase> cases;
  std::vector<int> Ns;
  std::vector<int> has_prism;
  int mixed = 0;
  cudaStream_t stream = nullptr;
  int device = 0, sms = 0;
  BatchCase *d_cases = nullptr;
  BatchTask *d_tasks = nullptr;
  size_t d_tasks_cap = 0;
  double *d_dts = nullptr;
  BatchSync *d_sync = nullptr;
  int *h_status = nullptr;   // pinned: err, nonfinite
  int mode = 0;    // 0: one cooperative persistent kernel per stage; 1: per-case kernels in one graph
  std::vector<double> h_dts;
  int block = 256, blocks_per_sm = 1, grid = 0;
  size_t smem = 0;
  int phase_begin[6] = {0};
  int n_phases = 0;
  long long spin_limit = 20000000;   // ~ 2.5 s of 128 ns sleeps per barrier wait
  int debug_skip = -1;
  cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
  fr_status poisoned = FR_OK;
  std::string err;
  int64_t n_points = 0;
};

static std::string g_batch_create_error;

static fr_status bfail(fr_batch *b, fr_status st, const std::string &msg) {
  if (b) {
    b->err = msg;
    if (st == FR_ECUDA || st == FR_ETIMEOUT) b->poisoned = st;
  } else {
    g_batch_create_error = msg;
  }
  return st;
}

static void drop_graphs(fr_batch *b) {
  for (auto &g : b->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// Task lists for one block size: phases interp | [bc prepare] | volume | interface (+ bc flux) | correct.
static std::vector<BatchTask> build_tasks(fr_batch *b, int block, int *phase_begin, int *n_phases) {
  std::vector<int> order(b->cases.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->Ns[x] > b->Ns[y]; });
  std::vector<BatchTask> t;
  auto chunks = [&](int cs, int kind, int64_t begin, int64_t end, int64_t step) {
    for (int64_t a = begin; a < end; a += step) t.push_back({cs, kind, a, std::min(end, a + step)});
  };
  bool any_bc = false;
  for (const BatchCase &c : b->cases) any_bc |= c.m.n_if > c.m.n_interior;
  int np = 0;
  phase_begin[np++] = 0;
  for (int cs : order) {
    const DevMesh &m = b->cases[cs].m;
    chunks(cs, TASK_INTERP, 0, m.E * 6 * m.Nf, block);
    chunks(cs, TASK_PRISM_INTERP, 0, m.Ep * 5 * m.Nf, block);
  }
  if (any_bc) {
    phase_begin[np++] = (int)t.size();
    for (int cs : order) {
      const DevMesh &m = b->cases[cs].m;
      chunks(cs, TASK_BC_PREPARE, 0, (m.n_if - m.n_interior) * m.Nf, block);
    }
  }
  phase_begin[np++] = (int)t.size();
  for (int cs : order) {
    const DevMesh &m = b->cases[cs].m;
    chunks(cs, TASK_VOLUME, 0, m.E, batch_elems_per_block(m.N, block));
    chunks(cs, TASK_PRISM_VOLUME, 0, m.Ep, batch_prism_elems_per_block(m.N, block));
  }
  phase_begin[np++] = (int)t.size();
  for (int cs : order) {
    const DevMesh &m = b->cases[cs].m;
    chunks(cs, TASK_IFACE, 0, m.n_interior * m.Nf, block);
    chunks(cs, TASK_BC_FLUX, 0, (m.n_if - m.n_interior) * m.Nf, block);
  }
  phase_begin[np++] = (int)t.size();
  for (int cs : order) {
    const DevMesh &m = b->cases[cs].m;
    chunks(cs, TASK_CORRECT, 0, m.E * m.Np, block);
    chunks(cs, TASK_PRISM_CORRECT, 0, m.Ep * m.Npp, block);
  }
  phase_begin[np] = (int)t.size();
  *n_phases = np;
  return t;
}

// Configure for a block size and resident blocks per SM (uploads the task list).
static fr_status configure(fr_batch *b, int block, int bps) {
  int phase_begin[6];
  int n_phases = 0;
  std::vector<BatchTask> tasks = build_tasks(b, block, phase_begin, &n_phases);
  const size_t smem = batch_smem_bytes(b->Ns.data(), b->has_prism.data(), (int)b->Ns.size(), block, b->mixed);
  int occ = 0;
  cudaError_t e = batch_occupancy(b->mixed, block, smem, &occ);
  if (e != cudaSuccess) return bfail(b, FR_ECUDA, std::string("batch occupancy: ") + cudaGetErrorString(e));
  if (occ < 1) return bfail(b, FR_EUNSUPPORTED, "batch kernel does not fit on an SM with this block size");
  bps = std::max(1, std::min(bps, occ));
  if (tasks.size() > b->d_tasks_cap) {
    if (b->d_tasks) cudaFree(b->d_tasks);
    b->d_tasks = nullptr;
    e = cudaMalloc((void **)&b->d_tasks, tasks.size() * sizeof(BatchTask));
    if (e != cudaSuccess) return bfail(b, FR_ENOMEM, "task list allocation failed");
    b->d_tasks_cap = tasks.size();
  }
  e = cudaMemcpyAsync(b->d_tasks, tasks.data(), tasks.size() * sizeof(BatchTask), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, FR_ECUDA, std::string("task upload: ") + cudaGetErrorString(e));
  std::memcpy(b->phase_begin, phase_begin, sizeof(phase_begin));
  b->n_phases = n_phases;
  b->block = block;
  b->blocks_per_sm = bps;
  b->grid = bps * b->sms;
  b->smem = smem;
  drop_graphs(b);
  return FR_OK;
}

static cudaError_t enqueue_stage(fr_batch *b, int stage) {
  if (b->mode == 1) {
    // Every case's own specialised kernels, back to back on the stream.
    for (size_t i = 0; i < b->cases.size(); ++i) {
      cudaError_t e = launch_residual(b->cases[i].m, b->cases[i].ph, MODE_RK, stage, b->h_dts[i], nullptr, b->stream);
      if (e != cudaSuccess) return e;
    }
    return stage == 3 ? launch_gather_flags(b->d_cases, (int)b->cases.size(), b->d_sync, b->stream) : cudaSuccess;
  }
  BatchLaunch L;
  L.cases = b->d_cases;
  L.tasks = b->d_tasks;
  std::memcpy(L.phase_begin, b->phase_begin, sizeof(L.phase_begin));
  L.n_phases = b->n_phases;
  L.stage = stage;
  L.dts = b->d_dts;
  L.sync = b->d_sync;
  L.spin_limit = b->spin_limit;
  L.debug_skip_block = b->debug_skip;
  // Task counters and the barrier start at zero; the error and non-finite words persist until
  // the host reads them.
  cudaError_t e = cudaMemsetAsync(b->d_sync, 0, offsetof(BatchSync, err), b->stream);
  if (e != cudaSuccess) return e;
  return launch_batch_stage(L, b->mixed, b->block, b->grid, b->smem, b->stream);
}

static fr_status check_batch(fr_batch *b) {
  if (!b) return FR_EINVAL;
  return b->poisoned;
}

extern "C" fr_status fr_batch_create(fr_mesh *const *meshes, int32_t n, fr_batch **out) {
  if (!out) return bfail(nullptr, FR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!meshes || n < 1) return bfail(nullptr, FR_EINVAL, "no meshes");
  fr_batch *b = new (std::nothrow) fr_batch();
  if (!b) return bfail(nullptr, FR_ENOMEM, "host allocation failed");
  for (int i = 0; i < n; ++i) {
    BatchCase c;
    cudaStream_t st;
    int dev;
    fr_status s = frx_mesh_view(meshes[i], &c.m, &c.ph, &st, &dev);
    if (s != FR_OK) {
      delete b;
      return bfail(nullptr, s == FR_EINVAL ? FR_EINVAL : s, "a mesh is NULL or poisoned");
    }
    if (c.ph.closure) {
      delete b;
      return bfail(nullptr, FR_EUNSUPPORTED, "meshes with the eddy-viscosity closure cannot be batched");
    }
    if (c.m.tc || c.m.vf32) {
      delete b;
      return bfail(nullptr, FR_EUNSUPPORTED,
                   "FR_PREC_MIXED_TC and FR_PREC_MIXED_VF32 meshes are not batched (use FR_PREC_MIXED)");
    }
    if (frx_mesh_has_halo(meshes[i])) {
      delete b;
      return bfail(nullptr, FR_EUNSUPPORTED, "parts that share interfaces with other parts cannot be batched");
    }
    if (c.ph.vc_basis) {
      delete b;
      return bfail(nullptr, FR_EUNSUPPORTED, "meshes with a correction function c != 0 cannot be batched");
    }
    if (i == 0) {
      b->mixed = c.m.mixed;
      b->stream = st;
      b->device = dev;
    } else if (c.m.mixed != b->mixed || st != b->stream || dev != b->device) {
      delete b;
      return bfail(nullptr, FR_EINVAL, "batched meshes must share precision, stream and device");
    }
    b->meshes.push_back(meshes[i]);
    b->cases.push_back(c);
    b->Ns.push_back(c.m.N);
    b->has_prism.push_back(c.m.Ep > 0 ? 1 : 0);
    b->n_points += c.m.E * c.m.Np + c.m.Ep * c.m.Npp;
  }
  cudaError_t e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_cases, sizeof(BatchCase) * n);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_dts, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_sync, sizeof(BatchSync));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_status, 2 * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_cases, b->cases.data(), sizeof(BatchCase) * n, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_dts, 0, sizeof(double) * n, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_sync, 0, sizeof(BatchSync), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    std::string msg = std::string("batch setup: ") + cudaGetErrorString(e);
    fr_batch_free(b);
    return bfail(nullptr, FR_ECUDA, msg);
  }
  int maxN = 0;
  for (int N : b->Ns) maxN = std::max(maxN, N);
  fr_status s = configure(b, maxN >= 7 ? 512 : 256, 1);
  if (s != FR_OK) {
    std::string msg = b->err;
    fr_batch_free(b);
    return bfail(nullptr, s, msg);
  }
  *out = b;
  return FR_OK;
}

extern "C" fr_status fr_batch_set_dt(fr_batch *b, const double *dt_host) {
  fr_status st = check_batch(b);
  if (st) return st;
  if (!dt_host) return bfail(b, FR_EINVAL, "dt is NULL");
  for (size_t i = 0; i < b->cases.size(); ++i)
    if (!(dt_host[i] > 0.0) || !std::isfinite(dt_host[i])) return bfail(b, FR_EINVAL, "dt must be positive and finite");
  cudaError_t e = cudaMemcpyAsync(b->d_dts, dt_host, sizeof(double) * b->cases.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, FR_ECUDA, std::string("dt upload: ") + cudaGetErrorString(e));
  b->h_dts.assign(dt_host, dt_host + b->cases.size());
  drop_graphs(b);   // the per-case mode bakes dt into its graph
  return FR_OK;
}

static fr_status read_status(fr_batch *b) {
  cudaError_t e = cudaMemcpyAsync(b->h_status, &b->d_sync->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, FR_ECUDA, std::string("batch stage: ") + cudaGetErrorString(e));
  const int err = b->h_status[0], nonfinite = b->h_status[1];
  if (err || nonfinite) {
    cudaMemsetAsync(&b->d_sync->err, 0, 2 * sizeof(int), b->stream);
    cudaStreamSynchronize(b->stream);
  }
  if (err) {
    for (fr_mesh *m : b->meshes) frx_mesh_fail(m, FR_ETIMEOUT, "a batched stage gave up waiting at a grid barrier");
    return bfail(b, FR_ETIMEOUT, "a grid-barrier wait exceeded its limit; the batch is unusable");
  }
  if (nonfinite) return bfail(b, FR_ENONFINITE, "non-finite value in an updated state");
  return FR_OK;
}

extern "C" fr_status fr_batch_rk_stage(fr_batch *b, int32_t stage, double t) {
  (void)t;
  fr_status st = check_batch(b);
  if (st) return st;
  if (stage < 0 || stage > 3) return bfail(b, FR_EINVAL, "stage must be 0..3");
  cudaError_t e;
  if (b->mode == 1 && b->h_dts.size() != b->cases.size()) return bfail(b, FR_EINVAL, "call fr_batch_set_dt first");
  if (b->stream != nullptr && b->debug_skip < 0) {
    // One graph per stage on a capturable (non-default) stream.
    if (!b->graph[stage]) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t le = enqueue_stage(b, stage);
        e = cudaStreamEndCapture(b->stream, &g);
        if (le != cudaSuccess) e = le;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[stage], g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return bfail(b, FR_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphLaunch(b->graph[stage], b->stream);
  } else {
    e = enqueue_stage(b, stage);
  }
  if (e != cudaSuccess) return bfail(b, FR_ECUDA, std::string("batch stage launch: ") + cudaGetErrorString(e));
  if (stage == 3 || b->debug_skip >= 0) return read_status(b);
  return FR_OK;
}

// Restore every case to U_n (a tuning run advanced their stage states).
static cudaError_t restore_states(fr_batch *b) {
  for (const BatchCase &c : b->cases) {
    const size_t bytes = ((size_t)c.m.E * c.m.Np + (size_t)c.m.Ep * c.m.Npp) * 5 * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(c.m.Q, c.m.Un, bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = launch_state_copy(c.m, b->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaStreamSynchronize(b->stream);
}

extern "C" fr_status fr_batch_tune(fr_batch *b) {
  fr_status st = check_batch(b);
  if (st) return st;
  int maxN = 0;
  for (int N : b->Ns) maxN = std::max(maxN, N);
  const int blocks[2] = {256, 512};
  float best_ms = 1e30f;
  int best_block = b->block, best_bps = b->blocks_per_sm;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int bi = 0; bi < 2; ++bi) {
    const int block = blocks[bi];
    if (maxN >= 7 && block < 512) continue;
    for (int bps = 1; bps <= 4; ++bps) {
      if (configure(b, block, bps) != FR_OK) {
        b->poisoned = FR_OK;
        continue;
      }
      if (b->blocks_per_sm != bps) continue;   // occupancy clamped: already measured
      cudaError_t e = enqueue_stage(b, 0);
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = enqueue_stage(b, 0);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return bfail(b, FR_ECUDA, std::string("batch tuning: ") + cudaGetErrorString(e));
      }
      if (ms < best_ms) {
        best_ms = ms;
        best_block = block;
        best_bps = bps;
      }
    }
  }
  // Per-case kernels (the same work as separate launches; captured into one graph per stage).
  int best_mode = 0;
  {
    std::vector<double> saved = b->h_dts;
    if (b->h_dts.size() != b->cases.size()) b->h_dts.assign(b->cases.size(), 0.0);
    b->mode = 1;
    cudaError_t e = enqueue_stage(b, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = enqueue_stage(b, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    b->mode = 0;
    b->h_dts = saved;
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return bfail(b, FR_ECUDA, std::string("batch tuning: ") + cudaGetErrorString(e));
    }
    if (ms < best_ms) {
      best_ms = ms;
      best_mode = 1;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  fr_status s = read_status(b);
  if (s != FR_OK) return s;
  s = configure(b, best_block, best_bps);
  b->mode = best_mode;
  if (s != FR_OK) return s;
  cudaError_t e = restore_states(b);
  if (e != cudaSuccess) return bfail(b, FR_ECUDA, std::string("batch restore: ") + cudaGetErrorString(e));
  return FR_OK;
}

extern "C" fr_status fr_batch_query(const fr_batch *b, fr_batch_info *info) {
  if (!b || !info) return FR_EINVAL;
  info->n_cases = (int32_t)b->cases.size();
  info->block = b->block;
  info->grid = b->grid;
  info->blocks_per_sm = b->blocks_per_sm;
  info->n_points = b->n_points;
  info->smem_bytes = (int64_t)b->smem;
  info->n_tasks = b->phase_begin[b->n_phases];
  info->mode = b->mode;
  return FR_OK;
}

extern "C" fr_status fr_batch_select(fr_batch *b, int32_t mode) {
  fr_status st = check_batch(b);
  if (st) return st;
  if (mode != 0 && mode != 1) return bfail(b, FR_EINVAL, "mode must be 0 or 1");
  b->mode = mode;
  drop_graphs(b);
  return FR_OK;
}

extern "C" fr_status fr_batch_debug(fr_batch *b, int32_t skip_block, int64_t spin_limit) {
  fr_status st = check_batch(b);
  if (st) return st;
  if (spin_limit < 1) return bfail(b, FR_EINVAL, "spin limit must be positive");
  b->debug_skip = skip_block;
  b->spin_limit = spin_limit;
  b->mode = 0;
  drop_graphs(b);
  return FR_OK;
}

extern "C" void fr_batch_free(fr_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  if (b->d_cases) cudaFree(b->d_cases);
  if (b->d_tasks) cudaFree(b->d_tasks);
  if (b->d_dts) cudaFree(b->d_dts);
  if (b->d_sync) cudaFree(b->d_sync);
  if (b->h_status) cudaFreeHost(b->h_status);
  delete b;
}

extern "C" const char *fr_batch_last_error(const fr_batch *b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}
