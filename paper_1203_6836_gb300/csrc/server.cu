// Serving runtime: continuous batching of XL-BOMD step requests from many
// trajectories of uneven size on one GPU.
//
// Every admitted trajectory keeps its whole state resident in one device
// allocation (R, v, F, the n history, q, H, D, gamma, mu and the workspace of
// its density solve), so a step needs no allocation and no host copy of the
// state.  Admission is by device-memory footprint: trajectories are admitted
// in arrival order while the sum of the admitted footprints stays within the
// budget; the rest wait and are admitted when a retired trajectory frees its
// memory.  Admission runs the initial SCF (xlbomd_init) and captures one step
// into a CUDA graph (the chemical-potential loop of dm_fermi becomes a while
// node), so a step request costs one graph launch.
//
// Requests are served in submission order, at most one step in flight per
// trajectory (its next step needs the previous one), on up to max_slots
// streams: a request is launched as soon as its trajectory is idle and a
// slot is free, while steps of other trajectories are still on the GPU, so
// small steps fill the SMs that a large one leaves idle.  Completion is seen
// by querying each slot's event; the step's energies and solver status come
// back by one small asynchronous copy into pinned memory.
//
// Trajectory memory comes from the stream-ordered allocator on the runtime's
// own stream (cudaMallocAsync / cudaFreeAsync), so admitting or retiring a
// trajectory does not synchronise the device under the steps in flight; the
// pinned completion buffers are kept in a free list.  Admission itself (the
// initial SCF) runs on the host and holds up dispatch while it lasts.  A
// trajectory whose admission fails gets its queued requests back as
// completions with the failure status.

#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <deque>
#include <list>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

enum TrajState { T_WAITING = 0, T_IDLE = 1, T_RUNNING = 2, T_RETIRED = 3, T_FAILED = 4 };

struct Request {
  int64_t id;
  int traj;
  double t_submit;
};

struct Traj {
  int natoms = 0, norb = 0;
  double n_occ = 0, box = 0;
  std::vector<int32_t> types, orb_off;
  std::vector<double> R0, v0, mass;
  size_t footprint = 0;
  int state = T_WAITING;
  bool retire = false;
  int queued = 0;  // submitted requests not yet launched
  void* mem = nullptr;
  tb_md_state st{};
  cudaGraphExec_t exec = nullptr;
  double* host = nullptr;  // pinned: energies[8], then the solver report
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;
  bool busy = false;
  Request req{};
  double t_launch = 0;
};

constexpr size_t kAlign = 1024;
constexpr size_t kHostDoubles = 8 + 16;  // energies + a report (<= 128 bytes)
static_assert(sizeof(tb_sp2_report) <= 16 * sizeof(double) && sizeof(tb_fermi_report) <= 16 * sizeof(double),
              "solver report does not fit the pinned completion buffer");

inline size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t R, v, F, mass, hist, q, H, D, gamma, energies, sp2rep, fermirep, mu, types, orb, ws, ws_bytes, total;
};

}  // namespace

struct tb_server {
  tb_ctx* ctx = nullptr;
  tb_params p{};
  tb_server_opts o{};
  std::vector<Traj> trajs;
  std::vector<Slot> slots;
  std::deque<int> waiting;  // trajectories awaiting admission, FIFO
  std::list<Request> pending;  // submitted, not launched, in submission order
  std::deque<tb_completion> failed;  // requests of trajectories whose admission failed
  std::vector<double*> host_pool;    // free pinned completion buffers
  size_t used = 0;
  int64_t next_id = 0, submitted = 0, completed = 0;
  cudaStream_t init_s = nullptr;
  Clock::time_point t0;
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

int layout_for(tb_server* sv, int N, int n, Layout* L) {
  size_t ws = 0;
  if (sv->o.kT > 0.0) {
    if (dm_fermi_workspace_size(n, &sv->o.fermi, &ws)) return tb_fail(sv->ctx, TB_ERR_ARG, "invalid fermi options");
  } else if (dm_sp2_workspace_size(n, &sv->o.sp2, &ws)) {
    return tb_fail(sv->ctx, TB_ERR_ARG, "invalid sp2 options");
  }
  const int K = sv->o.xl.K;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o += up(bytes);
    return r;
  };
  L->R = take(sizeof(double) * 3 * N);
  L->v = take(sizeof(double) * 3 * N);
  L->F = take(sizeof(double) * 3 * N);
  L->mass = take(sizeof(double) * N);
  L->hist = take(sizeof(double) * (size_t)(K + 1) * N);
  L->q = take(sizeof(double) * N);
  L->H = take(sizeof(double) * (size_t)n * n);
  L->D = take(sizeof(double) * (size_t)n * n);
  L->gamma = take(sizeof(double) * (size_t)N * N);
  L->energies = take(sizeof(double) * 8);
  L->sp2rep = take(sizeof(tb_sp2_report));
  L->fermirep = take(sizeof(tb_fermi_report));
  L->mu = take(4 * sizeof(double));
  L->types = take(sizeof(int32_t) * N);
  L->orb = take(sizeof(int32_t) * (N + 1));
  L->ws = take(ws);
  L->ws_bytes = ws;
  L->total = o + kAlign;  // one alignment unit of slack (the block is aligned in admit)
  return TB_OK;
}

// Allocate, upload, SCF-initialise and capture the step graph of trajectory t.
int admit(tb_server* sv, int t) {
  Traj& T = sv->trajs[t];
  tb_ctx* ctx = sv->ctx;
  Layout L{};
  int rc = layout_for(sv, T.natoms, T.norb, &L);
  if (rc) return rc;
  cudaStream_t s = sv->init_s;
  // the pool guarantees less than the 1024-byte alignment the workspace
  // needs: the layout holds one alignment unit of slack, and the state starts
  // at the first boundary
  TB_CUDA_TRY(ctx, cudaMallocAsync(&T.mem, L.total, s));
  sv->used += T.footprint;
  if (!sv->host_pool.empty()) {
    T.host = sv->host_pool.back();
    sv->host_pool.pop_back();
  } else {
    TB_CUDA_TRY(ctx, cudaHostAlloc((void**)&T.host, sizeof(double) * kHostDoubles, cudaHostAllocDefault));
  }
  char* b = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(T.mem) + kAlign - 1) & ~uintptr_t(kAlign - 1));
  const int N = T.natoms;
  TB_CUDA_TRY(ctx, cudaMemsetAsync(b, 0, L.total - kAlign, s));
  TB_CUDA_TRY(ctx, cudaMemcpyAsync(b + L.R, T.R0.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
  TB_CUDA_TRY(ctx, cudaMemcpyAsync(b + L.v, T.v0.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
  TB_CUDA_TRY(ctx, cudaMemcpyAsync(b + L.mass, T.mass.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
  TB_CUDA_TRY(ctx, cudaMemcpyAsync(b + L.types, T.types.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
  TB_CUDA_TRY(ctx,
              cudaMemcpyAsync(b + L.orb, T.orb_off.data(), sizeof(int32_t) * (N + 1), cudaMemcpyHostToDevice, s));
  const double nan4[4] = {NAN, NAN, NAN, NAN};
  TB_CUDA_TRY(ctx, cudaMemcpyAsync(b + L.mu, nan4, sizeof(nan4), cudaMemcpyHostToDevice, s));
  tb_md_state& st = T.st;
  st = tb_md_state{};
  st.sys.natoms = N;
  st.sys.norb = T.norb;
  st.sys.types = reinterpret_cast<const int32_t*>(b + L.types);
  st.sys.orb_off = reinterpret_cast<const int32_t*>(b + L.orb);
  st.sys.box = T.box;
  st.n_occ = T.n_occ;
  st.R = reinterpret_cast<double*>(b + L.R);
  st.v = reinterpret_cast<double*>(b + L.v);
  st.F = reinterpret_cast<double*>(b + L.F);
  st.mass = reinterpret_cast<const double*>(b + L.mass);
  st.n_hist = reinterpret_cast<double*>(b + L.hist);
  st.q = reinterpret_cast<double*>(b + L.q);
  st.H = reinterpret_cast<double*>(b + L.H);
  st.D = reinterpret_cast<double*>(b + L.D);
  st.gamma = reinterpret_cast<double*>(b + L.gamma);
  st.energies = reinterpret_cast<double*>(b + L.energies);
  st.sp2_report = reinterpret_cast<tb_sp2_report*>(b + L.sp2rep);
  st.workspace = b + L.ws;
  st.workspace_bytes = L.ws_bytes;
  st.kT = sv->o.kT;
  st.fermi = sv->o.fermi;
  st.mu = reinterpret_cast<double*>(b + L.mu);
  st.fermi_report = reinterpret_cast<tb_fermi_report*>(b + L.fermirep);
  int scf_iters = 0;
  rc = xlbomd_init(ctx, &sv->p, &st, &sv->o.xl, &sv->o.sp2, sv->o.scf_tol, sv->o.scf_max_iter, &scf_iters, s);
  if (rc) return rc;
  // one step, captured on the init stream (thread-local capture mode)
  cudaGraph_t g = nullptr;
  TB_CUDA_TRY(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  rc = xlbomd_step(ctx, &sv->p, &st, &sv->o.xl, &sv->o.sp2, s);
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return tb_fail(ctx, TB_ERR_CUDA, "step capture: %s", cudaGetErrorString(e));
  st.step = 0;
  const cudaError_t ei = cudaGraphInstantiate(&T.exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return tb_fail(ctx, TB_ERR_CUDA, "step graph instantiate: %s", cudaGetErrorString(ei));
  TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  T.state = T_IDLE;
  return TB_OK;
}

// Give back a trajectory's memory: its device block to the stream-ordered
// pool (after the work already on the runtime's stream; its own steps have
// completed), its pinned buffer to the free list.
void release(tb_server* sv, int t) {
  Traj& T = sv->trajs[t];
  if (T.exec) cudaGraphExecDestroy(T.exec);
  if (T.mem) cudaFreeAsync(T.mem, sv->init_s);
  if (T.host) sv->host_pool.push_back(T.host);
  if (T.mem) sv->used -= T.footprint;
  T.exec = nullptr;
  T.mem = nullptr;
  T.host = nullptr;
}

// Admit waiting trajectories in order while their footprint fits.
int admit_waiting(tb_server* sv) {
  while (!sv->waiting.empty()) {
    const int t = sv->waiting.front();
    Traj& T = sv->trajs[t];
    if (T.retire) {  // retired before it was admitted
      sv->waiting.pop_front();
      T.state = T_RETIRED;
      continue;
    }
    if (sv->used + T.footprint > sv->o.hbm_budget) break;
    sv->waiting.pop_front();
    const int rc = admit(sv, t);
    if (rc) {
      release(sv, t);
      T.state = T_FAILED;
      // its queued requests can never run: hand them back as failed completions
      for (auto it = sv->pending.begin(); it != sv->pending.end();) {
        if (it->traj != t) {
          ++it;
          continue;
        }
        tb_completion c{};
        c.request = it->id;
        c.traj = t;
        c.status = rc;
        c.t_submit = it->t_submit;
        c.t_launch = c.t_done = sv->now();
        sv->failed.push_back(c);
        T.queued -= 1;
        it = sv->pending.erase(it);
      }
      return rc;
    }
  }
  return TB_OK;
}

// Free the memory of retired idle trajectories.
void reap(tb_server* sv) {
  for (size_t t = 0; t < sv->trajs.size(); ++t) {
    Traj& T = sv->trajs[t];
    if (T.retire && T.state == T_IDLE && T.queued == 0) {
      release(sv, (int)t);
      T.state = T_RETIRED;
    }
  }
}

int launch(tb_server* sv, Slot& sl, const Request& r) {
  tb_ctx* ctx = sv->ctx;
  Traj& T = sv->trajs[r.traj];
  sl.busy = true;
  sl.req = r;
  sl.t_launch = sv->now();
  TB_CUDA_TRY(ctx, cudaEventRecord(sl.start, sl.s));
  TB_CUDA_TRY(ctx, cudaGraphLaunch(T.exec, sl.s));
  TB_CUDA_TRY(ctx, cudaMemcpyAsync(T.host, T.st.energies, sizeof(double) * 8, cudaMemcpyDeviceToHost, sl.s));
  if (sv->o.kT > 0.0)
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(T.host + 8, T.st.fermi_report, sizeof(tb_fermi_report),
                                     cudaMemcpyDeviceToHost, sl.s));
  else
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(T.host + 8, T.st.sp2_report, sizeof(tb_sp2_report), cudaMemcpyDeviceToHost,
                                     sl.s));
  TB_CUDA_TRY(ctx, cudaEventRecord(sl.done, sl.s));
  T.state = T_RUNNING;
  T.queued -= 1;
  return TB_OK;
}

// Launch pending requests of idle admitted trajectories, oldest first.
int dispatch(tb_server* sv) {
  size_t free_slot = 0;
  for (auto it = sv->pending.begin(); it != sv->pending.end();) {
    while (free_slot < sv->slots.size() && sv->slots[free_slot].busy) ++free_slot;
    if (free_slot == sv->slots.size()) break;
    Traj& T = sv->trajs[it->traj];
    if (T.state != T_IDLE) {
      ++it;
      continue;
    }
    const int rc = launch(sv, sv->slots[free_slot], *it);
    if (rc) return rc;
    it = sv->pending.erase(it);
  }
  return TB_OK;
}

// Collect finished slots into out[]; returns the count.
int collect(tb_server* sv, tb_completion* out, int max_out, int* n_out) {
  int k = 0;
  while (!sv->failed.empty() && k < max_out) {
    out[k++] = sv->failed.front();
    sv->failed.pop_front();
    sv->completed += 1;
  }
  for (Slot& sl : sv->slots) {
    if (!sl.busy || k >= max_out) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return tb_fail(sv->ctx, TB_ERR_CUDA, "step: %s", cudaGetErrorString(q));
    const double t_done = sv->now();
    Traj& T = sv->trajs[sl.req.traj];
    tb_completion& c = out[k++];
    c = tb_completion{};
    c.request = sl.req.id;
    c.traj = sl.req.traj;
    c.status = reinterpret_cast<const int*>(T.host + 8)[0];
    c.solver_iters = reinterpret_cast<const int*>(T.host + 8)[1];  // iters / mu_iters
    c.solver_m = sv->o.kT > 0.0 ? reinterpret_cast<const int*>(T.host + 8)[2] : 0;  // tb_fermi_report.m
    c.step = (int64_t)T.host[7];
    c.t_submit = sl.req.t_submit;
    c.t_launch = sl.t_launch;
    c.t_done = t_done;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, sl.start, sl.done) == cudaSuccess) c.gpu_ms = ms;
    for (int i = 0; i < 8; ++i) c.energies[i] = T.host[i];
    sl.busy = false;
    T.state = T_IDLE;
    T.st.step += 1;
    sv->completed += 1;
  }
  *n_out = k;
  return TB_OK;
}

int progress(tb_server* sv, tb_completion* out, int max_out, int* n_out) {
  int rc = collect(sv, out, max_out, n_out);
  if (rc) return rc;
  reap(sv);
  if ((rc = admit_waiting(sv))) return rc;
  return dispatch(sv);
}

bool any_busy(const tb_server* sv) {
  for (const Slot& sl : sv->slots)
    if (sl.busy) return true;
  return false;
}

int do_submit(tb_server* sv, int traj, double t_submit, int64_t* id) {
  if (traj < 0 || traj >= (int)sv->trajs.size()) return tb_fail(sv->ctx, TB_ERR_ARG, "no trajectory %d", traj);
  Traj& T = sv->trajs[traj];
  if (T.retire || T.state == T_RETIRED || T.state == T_FAILED)
    return tb_fail(sv->ctx, TB_ERR_ARG, "trajectory %d is retired or failed", traj);
  const Request r{sv->next_id++, traj, t_submit};
  sv->pending.push_back(r);
  T.queued += 1;
  sv->submitted += 1;
  if (id) *id = r.id;
  return TB_OK;
}

}  // namespace

extern "C" int tb_server_footprint(const tb_server* sv, int natoms, const int32_t* types, size_t* bytes) {
  if (!sv || !types || !bytes || natoms < 1) return TB_ERR_ARG;
  int n = 0;
  for (int i = 0; i < natoms; ++i) n += types[i] == TB_TYPE_O ? 4 : 1;
  Layout L{};
  const int rc = layout_for(const_cast<tb_server*>(sv), natoms, n, &L);
  if (rc) return rc;
  *bytes = L.total;
  return TB_OK;
}

extern "C" int tb_server_create(tb_ctx* ctx, const tb_params* p, const tb_server_opts* o, tb_server** out) {
  if (!ctx) return TB_ERR_ARG;
  if (!p || !o || !out) return tb_fail(ctx, TB_ERR_ARG, "null argument to tb_server_create");
  if (o->max_slots < 1 || o->max_slots > TB_SERVER_MAX_SLOTS)
    return tb_fail(ctx, TB_ERR_ARG, "max_slots = %d outside 1..%d", o->max_slots, TB_SERVER_MAX_SLOTS);
  if (o->xl.K < 1 || o->xl.K > TB_XL_KMAX || !(o->xl.dt > 0) || !(o->kT >= 0.0) || o->scf_max_iter < 1)
    return tb_fail(ctx, TB_ERR_ARG, "invalid XL-BOMD parameters, kT or scf_max_iter");
  *out = nullptr;
  tb_server* sv = new tb_server();
  sv->ctx = ctx;
  sv->p = *p;
  sv->o = *o;
  sv->t0 = Clock::now();
  auto fail = [&](int rc) {
    tb_server_destroy(sv);
    return rc;
  };
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(tb_fail(ctx, TB_ERR_CUDA, "cudaMemGetInfo"));
  if (sv->o.hbm_budget == 0) sv->o.hbm_budget = free_b / 10 * 9;
  if (cudaStreamCreateWithFlags(&sv->init_s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(tb_fail(ctx, TB_ERR_CUDA, "stream create"));
  sv->slots.resize(o->max_slots);
  for (Slot& sl : sv->slots) {
    if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sl.start) != cudaSuccess || cudaEventCreate(&sl.done) != cudaSuccess)
      return fail(tb_fail(ctx, TB_ERR_CUDA, "slot stream/event create"));
  }
  *out = sv;
  return TB_OK;
}

extern "C" int tb_server_destroy(tb_server* sv) {
  if (!sv) return TB_OK;
  for (Slot& sl : sv->slots) {
    if (sl.s) cudaStreamSynchronize(sl.s);
  }
  for (size_t t = 0; t < sv->trajs.size(); ++t) release(sv, (int)t);
  if (sv->init_s) cudaStreamSynchronize(sv->init_s);
  for (double* h : sv->host_pool) cudaFreeHost(h);
  for (Slot& sl : sv->slots) {
    if (sl.start) cudaEventDestroy(sl.start);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.s) cudaStreamDestroy(sl.s);
  }
  if (sv->init_s) cudaStreamDestroy(sv->init_s);
  delete sv;
  return TB_OK;
}

extern "C" int tb_server_add(tb_server* sv, int natoms, const int32_t* types, double box, const double* R0,
                             const double* v0, const double* mass, double n_occ, int* traj_out) {
  if (!sv) return TB_ERR_ARG;
  tb_ctx* ctx = sv->ctx;
  if (natoms < 1 || !types || !R0 || !v0 || !mass || !traj_out || !(box > 0))
    return tb_fail(ctx, TB_ERR_ARG, "invalid trajectory arguments");
  Traj T;
  T.natoms = natoms;
  T.box = box;
  T.n_occ = n_occ;
  T.types.assign(types, types + natoms);
  T.orb_off.resize(natoms + 1);
  int n = 0;
  for (int i = 0; i < natoms; ++i) {
    if (types[i] != TB_TYPE_O && types[i] != TB_TYPE_H) return tb_fail(ctx, TB_ERR_ARG, "bad atom type");
    T.orb_off[i] = n;
    n += types[i] == TB_TYPE_O ? 4 : 1;
  }
  T.orb_off[natoms] = n;
  T.norb = n;
  if (!(n_occ >= 0.0) || n_occ > n) return tb_fail(ctx, TB_ERR_ARG, "n_occ outside [0, n]");
  T.R0.assign(R0, R0 + 3 * (size_t)natoms);
  T.v0.assign(v0, v0 + 3 * (size_t)natoms);
  T.mass.assign(mass, mass + natoms);
  Layout L{};
  int rc = layout_for(sv, natoms, n, &L);
  if (rc) return rc;
  T.footprint = L.total;
  if (T.footprint > sv->o.hbm_budget)
    return tb_fail(ctx, TB_ERR_OOM, "trajectory footprint %zu bytes exceeds the budget %zu", T.footprint,
                   sv->o.hbm_budget);
  sv->trajs.push_back(std::move(T));
  const int t = (int)sv->trajs.size() - 1;
  sv->waiting.push_back(t);
  *traj_out = t;
  return admit_waiting(sv);
}

extern "C" int tb_server_submit(tb_server* sv, int traj, int64_t* request_out) {
  if (!sv) return TB_ERR_ARG;
  int rc = do_submit(sv, traj, sv->now(), request_out);
  if (rc) return rc;
  int n = 0;
  return progress(sv, nullptr, 0, &n);
}

extern "C" int tb_server_poll(tb_server* sv, int wait, tb_completion* out, int max_out, int* n_out) {
  if (!sv) return TB_ERR_ARG;
  if (!n_out || max_out < 0 || (max_out > 0 && !out)) return tb_fail(sv->ctx, TB_ERR_ARG, "bad poll output");
  *n_out = 0;
  for (;;) {
    int rc = progress(sv, out, max_out, n_out);
    if (rc) return rc;
    if (*n_out > 0 || !wait || max_out == 0 || !any_busy(sv)) return TB_OK;
    std::this_thread::yield();
  }
}

extern "C" int tb_server_retire(tb_server* sv, int traj) {
  if (!sv) return TB_ERR_ARG;
  if (traj < 0 || traj >= (int)sv->trajs.size()) return tb_fail(sv->ctx, TB_ERR_ARG, "no trajectory %d", traj);
  sv->trajs[traj].retire = true;
  int n = 0;
  return progress(sv, nullptr, 0, &n);
}

extern "C" int tb_server_read(tb_server* sv, int traj, double* R, double* v, double* q, double* n_t,
                              double* energies) {
  if (!sv) return TB_ERR_ARG;
  if (traj < 0 || traj >= (int)sv->trajs.size()) return tb_fail(sv->ctx, TB_ERR_ARG, "no trajectory %d", traj);
  Traj& T = sv->trajs[traj];
  if (T.state != T_IDLE) return tb_fail(sv->ctx, TB_ERR_ARG, "trajectory %d is not admitted and idle", traj);
  const int N = T.natoms;
  cudaStream_t s = sv->init_s;
  tb_ctx* ctx = sv->ctx;
  if (R) TB_CUDA_TRY(ctx, cudaMemcpyAsync(R, T.st.R, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s));
  if (v) TB_CUDA_TRY(ctx, cudaMemcpyAsync(v, T.st.v, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s));
  if (q) TB_CUDA_TRY(ctx, cudaMemcpyAsync(q, T.st.q, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  if (n_t) TB_CUDA_TRY(ctx, cudaMemcpyAsync(n_t, T.st.n_hist, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  if (energies) TB_CUDA_TRY(ctx, cudaMemcpyAsync(energies, T.st.energies, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
  TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return TB_OK;
}

extern "C" int tb_server_stats(const tb_server* sv, tb_server_counts* out) {
  if (!sv || !out) return TB_ERR_ARG;
  *out = tb_server_counts{};
  out->trajectories = (int)sv->trajs.size();
  for (const Traj& T : sv->trajs) {
    if (T.state == T_IDLE || T.state == T_RUNNING) out->admitted += 1;
    if (T.state == T_WAITING) out->waiting += 1;
    if (T.state == T_RUNNING) out->running += 1;
  }
  out->queued = (int)sv->pending.size();
  out->bytes_in_use = sv->used;
  out->budget = sv->o.hbm_budget;
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  return TB_OK;
}

extern "C" int tb_server_replay(tb_server* sv, int count, const double* arrival_s, const int* traj,
                                tb_completion* out) {
  if (!sv) return TB_ERR_ARG;
  if (count < 0 || (count > 0 && (!arrival_s || !traj || !out)))
    return tb_fail(sv->ctx, TB_ERR_ARG, "bad replay arguments");
  for (int i = 1; i < count; ++i)
    if (arrival_s[i] < arrival_s[i - 1]) return tb_fail(sv->ctx, TB_ERR_ARG, "arrival times must not decrease");
  for (int i = 0; i < count; ++i) {
    if (traj[i] < 0 || traj[i] >= (int)sv->trajs.size() || sv->trajs[traj[i]].retire)
      return tb_fail(sv->ctx, TB_ERR_ARG, "request %d names no live trajectory", i);
  }
  if (!sv->pending.empty() || any_busy(sv))
    return tb_fail(sv->ctx, TB_ERR_ARG, "replay needs a server with no request outstanding");
  {
    // free retired trajectories and admit what fits first: nothing retires
    // during the replay, so a trajectory not admitted now never runs in it
    int k = 0;
    int rc = progress(sv, nullptr, 0, &k);
    if (rc) return rc;
  }
  for (int i = 0; i < count; ++i) {
    const int st = sv->trajs[traj[i]].state;
    if (st != T_IDLE && st != T_RUNNING)
      return tb_fail(sv->ctx, TB_ERR_ARG, "request %d names trajectory %d, which is not admitted", i, traj[i]);
  }
  const int64_t first = sv->next_id;
  const double base = sv->now();
  std::vector<tb_completion> buf(sv->slots.size());
  int next = 0, done = 0;
  while (done < count) {
    const double t = sv->now() - base;
    while (next < count && arrival_s[next] <= t) {
      int64_t id = 0;
      int rc = do_submit(sv, traj[next], base + arrival_s[next], &id);
      if (rc) return rc;
      ++next;
    }
    int k = 0;
    int rc = progress(sv, buf.data(), (int)buf.size(), &k);
    if (rc) return rc;
    for (int j = 0; j < k; ++j) {
      const int64_t idx = buf[j].request - first;
      if (idx >= 0 && idx < count) {
        out[idx] = buf[j];
        ++done;
      }
    }
    if (k == 0) {
      if (next == count && !any_busy(sv) && sv->failed.empty())
        return tb_fail(sv->ctx, TB_ERR_ARG, "replay stalled: %d of %d requests cannot run", count - done, count);
      std::this_thread::yield();
    }
  }
  return TB_OK;
}
