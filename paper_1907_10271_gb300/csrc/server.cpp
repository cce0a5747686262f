// Request loop with continuous batching on one GPU, and the selective refinement of
// Sec. 2.4 (Algorithm 2) as a request kind, for the strip (mlmc.h) and the buckling
// panel (mlmc_panel.h) alike: a backend supplies the per-worker contexts, the batch
// solve, the footprint of a solve and the failure quantity.
//
// Host side only: a FIFO of pending requests (escalations of selective-refinement
// samples go to its front), `workers` threads each owning an mlmc context on its own
// non-blocking CUDA stream. A free worker takes the oldest pending requests whose
// footprint fits its share of the device-memory budget (at most max_batch), runs them
// as one mlmc_solve_batch, and feeds the results back: SOLVE requests complete,
// SELECTIVE requests either stop (the stopping test of Eq. testFailure with the
// sample bias estimate of Eq. sampleBias) or re-enter the queue on the next mesh.
// Workspaces are reserved to the share up front, so serving allocates nothing. With
// carry_iterates, a SELECTIVE sample that may escalate takes a slot of a per-mesh
// pool (allocated at creation) for its final iterate on the mesh it is solving; its
// next mesh starts from that iterate (nested iteration) and gives the slot back.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mlmc_panel.h"
#include "engine.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
  mlmc_request req;
  Clock::time_point t0;
  int mesh = 0;   // SELECTIVE: next mesh to solve
  int solves = 0;
  double lambda[MLMC_SR_MAX_LEVELS] = {0};
  int iters[MLMC_SR_MAX_LEVELS] = {0};
  int carry = -1;   // pool slot on mesh - 1 holding the previous solve's iterate (or -1)
  int out = -1;     // pool slot on mesh receiving this solve's iterate (or -1)
};

// Fixed-size slots of device memory, one class per mesh, each one refinement iterate.
struct IteratePool {
  std::vector<double*> base;             // per mesh
  std::vector<int64_t> values;           // per mesh: doubles per slot
  std::vector<std::vector<int>> free;    // per mesh
  bool empty() const { return base.empty(); }
  double* at(int m, int slot) const { return base[m] + (int64_t)slot * values[m]; }
  int take(int m) {
    if (m >= (int)free.size() || free[m].empty()) return -1;
    const int k = free[m].back();
    free[m].pop_back();
    return k;
  }
  void give(int m, int slot) {
    if (slot >= 0) free[m].push_back(slot);
  }
  void release() {
    for (double* p : base)
      if (p) cudaFree(p);
    base.clear();
  }
};

// What a request loop needs from an engine.
struct Backend {
  virtual ~Backend() {}
  virtual int levels() const = 0;
  virtual double m_alpha_minus_one() const = 0;   // m^alpha - 1 of the bias estimate
  virtual int quantity() const = 0;               // index of the selective-refinement quantity
  virtual bool fails_below() const = 0;           // failure is lambda < lambda* (else >)
  virtual double footprint(int mesh) const = 0;   // device bytes of one solve on mesh
  virtual bool carries() const = 0;               // starting iterates across escalations
  virtual int64_t iterate_values(int mesh) const = 0;
  virtual mlmc_status add_worker(cudaStream_t st, double share, std::string& msg) = 0;
  // one batch on worker w; iters (host) per item; guess / out: see solve_batch_carry
  virtual mlmc_status solve(int w, const mlmc_item* items, int64_t n, double* q, int32_t* status,
                            const double* const* guess, double* const* out, int32_t* iters, std::string& msg) = 0;
};

struct StripBackend : Backend {
  mlmc_config cfg;
  std::vector<mlmc_ctx*> ctx;
  explicit StripBackend(const mlmc_config& c) : cfg(c) {}
  ~StripBackend() override {
    for (auto* c : ctx) mlmc_destroy(c);
  }
  int levels() const override { return cfg.levels; }
  double m_alpha_minus_one() const override { return std::pow(cfg.mlmc_m, cfg.mlmc_alpha) - 1.0; }
  int quantity() const override { return 1; }   // the centroid fibre stress
  bool fails_below() const override { return false; }
  double footprint(int mesh) const override { return mlmc::solve_bytes_per_sample(cfg, mesh); }
  bool carries() const override { return true; }
  int64_t iterate_values(int mesh) const override { return mlmc::iterate_values(cfg, mesh); }
  mlmc_status add_worker(cudaStream_t st, double share, std::string& msg) override {
    mlmc_ctx* c = nullptr;
    mlmc_status e = mlmc_create(&cfg, st, &c);
    if (e != MLMC_OK) {
      msg = std::string("worker context: ") + mlmc_last_error(nullptr);
      return e;
    }
    ctx.push_back(c);
    mlmc::set_graph_replay(c, false);   // every batch differs: no graph to reuse
    // the share, split like the footprint estimate: solver workspace and batch buffers
    e = mlmc::reserve_workspace(c, (size_t)(0.85 * share), (size_t)(0.15 * share));
    if (e != MLMC_OK) msg = std::string("worker workspace: ") + mlmc_last_error(c);
    return e;
  }
  mlmc_status solve(int w, const mlmc_item* items, int64_t n, double* q, int32_t* status, const double* const* guess,
                    double* const* out, int32_t* iters, std::string& msg) override {
    const mlmc_status s = mlmc::solve_batch_carry(ctx[w], items, n, q, status, guess, out, iters);
    if (s != MLMC_OK) msg = mlmc_last_error(ctx[w]);
    return s;
  }
};

// The buckling panel: the failure quantity is the critical load (quantity 0), failing
// below its threshold (Sec. 4.2); solves from scratch (no carried iterates); the
// engine's workspace is stream-ordered allocation per batch.
struct PanelBackend : Backend {
  mlmcp_config cfg;
  double m = 4.0, alpha = 1.0;
  std::vector<mlmcp_ctx*> ctx;
  PanelBackend(const mlmcp_config& c, double m_, double a_) : cfg(c), m(m_), alpha(a_) {}
  ~PanelBackend() override {
    for (auto* c : ctx) mlmcp_destroy(c);
  }
  int levels() const override { return cfg.levels; }
  double m_alpha_minus_one() const override { return std::pow(m, alpha) - 1.0; }
  int quantity() const override { return 0; }
  bool fails_below() const override { return true; }
  double footprint(int mesh) const override {
    // about 24 vectors of two columns of float4 per node over the hierarchy, the element
    // matrices and the coarsest inverse
    const double nodes = (double)((cfg.nx0 << mesh) + 1) * ((cfg.ny0 << mesh) + 1);
    return nodes * 2.0 * 16.0 * 24.0 + 200.0e3;
  }
  bool carries() const override { return false; }
  int64_t iterate_values(int) const override { return 0; }
  mlmc_status add_worker(cudaStream_t st, double, std::string& msg) override {
    mlmcp_ctx* c = nullptr;
    const mlmc_status e = mlmcp_create(&cfg, st, &c);
    if (e != MLMC_OK) {
      msg = std::string("worker context: ") + mlmcp_last_error(nullptr);
      return e;
    }
    ctx.push_back(c);
    return MLMC_OK;
  }
  mlmc_status solve(int w, const mlmc_item* items, int64_t n, double* q, int32_t* status, const double* const*,
                    double* const*, int32_t* iters, std::string& msg) override {
    const mlmc_status s = mlmcp_solve_batch(ctx[w], items, n, q, status);
    if (s != MLMC_OK) msg = mlmcp_last_error(ctx[w]);
    int32_t it = 0;
    mlmcp_last_iters(ctx[w], &it);
    for (int64_t k = 0; k < n; ++k) iters[k] = it;   // the batch's slowest sample
    return s;
  }
};

}  // namespace

struct mlmc_server {
  std::unique_ptr<Backend> be;
  mlmc_server_config scfg;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;
  std::deque<mlmc_result> done;
  int64_t outstanding = 0;
  bool stop = false;
  int64_t batches = 0, solves = 0;
  double in_flight = 0.0, peak = 0.0, share = 0.0;
  int device = 0;
  IteratePool pool;      // carried iterates (guarded by mu)
  char err[512] = {0};   // last failure message (stable storage for mlmc_server_last_error)

  void record_error(const std::string& m) {
    std::lock_guard<std::mutex> g(mu);
    std::strncpy(err, m.c_str(), sizeof(err) - 1);
  }

  // called with mu held
  void complete(const Pending& p, int32_t status, const double* q, int stop_level) {
    mlmc_result r;
    std::memset(&r, 0, sizeof(r));
    r.tag = p.req.tag;
    r.kind = p.req.kind;
    r.level = p.req.level;
    r.mesh_level = p.req.mesh_level;
    r.sample_id = p.req.sample_id;
    r.status = status;
    r.solves = p.solves;
    for (int j = 0; j < std::min(p.solves, MLMC_SR_MAX_LEVELS); ++j) r.pcg_iterations[j] = p.iters[j];
    if (q) {
      r.q[0] = q[0];
      r.q[1] = q[1];
    }
    if (p.req.kind == MLMC_REQ_SELECTIVE && status == 0) {
      r.stop_level = stop_level;
      for (int j = 0; j <= stop_level; ++j) r.lambda[j] = p.lambda[j];
      const int l = p.req.level;
      r.lambda_fine = p.lambda[stop_level];
      r.q_fine = fails(r.lambda_fine) ? 1 : 0;
      r.q_mesh0 = fails(p.lambda[0]) ? 1 : 0;
      if (l >= 1) {
        r.lambda_coarse = p.lambda[std::min(stop_level, l - 1)];
        r.q_coarse = fails(r.lambda_coarse) ? 1 : 0;
      }
    }
    r.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - p.t0).count();
    done.push_back(r);
    --outstanding;
  }

  bool fails(double lambda) const { return be->fails_below() ? lambda < scfg.threshold : lambda > scfg.threshold; }

  // Stopping test of a selective-refinement sample after its solve on mesh j.
  bool sr_stops(const Pending& p, int j) const {
    if (j >= p.req.level) return true;
    if (j < 1) return false;   // no bias estimate before two meshes
    const double lj = p.lambda[j], lp = p.lambda[j - 1];
    const double bias = std::fabs(lj - lp) / be->m_alpha_minus_one();
    const double bound = scfg.sr_factor * std::max(scfg.eps_rel * std::fabs(lj), bias);
    return std::fabs(lj - scfg.threshold) >= bound;
  }

  int mesh_of(const Pending& p) const { return p.req.kind == MLMC_REQ_SOLVE ? p.req.mesh_level : p.mesh; }

  void worker(int w) {
    cudaSetDevice(device);
    std::vector<Pending> batch;
    std::vector<mlmc_item> items;
    std::vector<double> q;
    std::vector<int32_t> st, its;
    std::vector<const double*> guess;
    std::vector<double*> outp;
    for (;;) {
      double bytes = 0.0;
      batch.clear();
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || !queue.empty(); });
        if (stop) return;
        while (!queue.empty() && (int64_t)batch.size() < scfg.max_batch) {
          const double b = be->footprint(mesh_of(queue.front()));
          if (batch.empty() && b > share) {   // can never fit
            Pending p = queue.front();
            queue.pop_front();
            if (p.carry >= 0) pool.give(p.mesh - 1, p.carry);
            complete(p, MLMC_ERR_OOM, nullptr, 0);
            cv_done.notify_all();
            continue;
          }
          if (bytes + b > share) break;
          bytes += b;
          batch.push_back(queue.front());
          queue.pop_front();
          // a sample that may escalate keeps this solve's iterate, if a slot is free
          Pending& p = batch.back();
          if (!pool.empty() && p.req.kind == MLMC_REQ_SELECTIVE && p.mesh < p.req.level) p.out = pool.take(p.mesh);
        }
        if (batch.empty()) continue;
        in_flight += bytes;
        peak = std::max(peak, in_flight);
      }
      items.resize(batch.size());
      guess.assign(batch.size(), nullptr);
      outp.assign(batch.size(), nullptr);
      for (size_t k = 0; k < batch.size(); ++k) {
        const Pending& p = batch[k];
        items[k].level = p.req.level;
        items[k].mesh_level = mesh_of(p);
        items[k].sample_id = p.req.sample_id;
        if (p.carry >= 0) guess[k] = pool.at(p.mesh - 1, p.carry);
        if (p.out >= 0) outp[k] = pool.at(p.mesh, p.out);
      }
      q.assign(2 * batch.size(), 0.0);
      st.assign(batch.size(), 0);
      its.assign(batch.size(), 0);
      std::string msg;
      const mlmc_status s = be->solve(w, items.data(), (int64_t)items.size(), q.data(), st.data(), guess.data(),
                                      outp.data(), its.data(), msg);
      if (s != MLMC_OK) record_error(msg);
      {
        std::lock_guard<std::mutex> g(mu);
        in_flight -= bytes;
        ++batches;
        solves += (int64_t)batch.size();
        std::vector<Pending> again;
        for (size_t k = 0; k < batch.size(); ++k) {
          Pending& p = batch[k];
          if (p.solves < MLMC_SR_MAX_LEVELS) p.iters[p.solves] = its[k];
          ++p.solves;
          const int32_t status = s != MLMC_OK ? (int32_t)s : st[k];
          // the previous mesh's iterate has been read; this solve's is kept only for an escalation
          if (p.carry >= 0) pool.give(p.mesh - 1, p.carry);
          p.carry = -1;
          if (status != 0 || p.req.kind == MLMC_REQ_SOLVE) {
            if (p.out >= 0) pool.give(p.mesh, p.out);
            p.out = -1;
            complete(p, status, &q[2 * k], 0);
            continue;
          }
          const int j = p.mesh;
          p.lambda[j] = q[2 * k + be->quantity()];
          if (sr_stops(p, j)) {
            if (p.out >= 0) pool.give(j, p.out);
            p.out = -1;
            complete(p, 0, &q[2 * k], j);
          } else {
            p.carry = p.out;
            p.out = -1;
            p.mesh = j + 1;
            again.push_back(p);
          }
        }
        // escalations go first, in their original order
        for (auto it = again.rbegin(); it != again.rend(); ++it) queue.push_front(*it);
        if (!again.empty()) cv_work.notify_all();
        cv_done.notify_all();
      }
    }
  }
};

namespace {
std::string g_server_error;
}

namespace {

// Common part of the two constructors: checks, the iterate pool (backends that carry),
// streams, worker contexts and threads.
mlmc_status start_server(std::unique_ptr<Backend> be, const mlmc_server_config* scfg, mlmc_server** out) {
  if (scfg->workers < 1 || scfg->workers > 64 || scfg->max_batch < 1 || !(scfg->hbm_budget_bytes > 0) ||
      !(scfg->sr_factor >= 1.0) || !(scfg->eps_rel >= 0.0) || be->levels() > MLMC_SR_MAX_LEVELS) {
    g_server_error = "bad server configuration";
    return MLMC_ERR_INVALID_ARG;
  }
  if (!(be->m_alpha_minus_one() > 0.0)) {
    g_server_error = "selective refinement needs mlmc_m > 1 and mlmc_alpha > 0";
    return MLMC_ERR_INVALID_ARG;
  }
  if (scfg->carry_iterates != 0 && scfg->carry_iterates != 1) {
    g_server_error = "carry_iterates must be 0 or 1";
    return MLMC_ERR_INVALID_ARG;
  }
  mlmc_server* s = new mlmc_server();
  s->be = std::move(be);
  s->scfg = *scfg;
  cudaGetDevice(&s->device);
  // carried iterates: 1/8 of the budget, split evenly over the meshes a sample can
  // escalate from (0 .. levels - 2), at most four slots per request a batch holds
  double pool_bytes = 0.0;
  const int levels = s->be->levels();
  if (scfg->carry_iterates && s->be->carries() && levels > 1) {
    const int meshes = levels - 1;
    const double per_mesh = scfg->hbm_budget_bytes / 8.0 / meshes;
    for (int m = 0; m < meshes; ++m) {
      const int64_t vals = s->be->iterate_values(m);
      const int64_t slots = std::min<int64_t>((int64_t)(per_mesh / (8.0 * vals)), 4 * scfg->max_batch * scfg->workers);
      double* base = nullptr;
      if (slots > 0 && cudaMalloc(&base, sizeof(double) * vals * slots) != cudaSuccess) {
        cudaGetLastError();
        s->pool.release();
        delete s;
        g_server_error = "iterate pool allocation failed";
        return MLMC_ERR_OOM;
      }
      s->pool.base.push_back(base);
      s->pool.values.push_back(vals);
      s->pool.free.emplace_back();
      for (int64_t k = slots - 1; k >= 0; --k) s->pool.free.back().push_back((int)k);
      pool_bytes += 8.0 * vals * slots;
    }
  }
  s->share = (scfg->hbm_budget_bytes - pool_bytes) / scfg->workers;
  for (int w = 0; w < scfg->workers; ++w) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      g_server_error = "stream creation failed";
      mlmc_server_destroy(s);
      return MLMC_ERR_CUDA;
    }
    s->streams.push_back(st);
    std::string msg;
    const mlmc_status e = s->be->add_worker(st, s->share, msg);
    if (e != MLMC_OK) {
      g_server_error = msg;
      mlmc_server_destroy(s);
      return e;
    }
  }
  for (int w = 0; w < scfg->workers; ++w) s->threads.emplace_back([s, w] { s->worker(w); });
  *out = s;
  return MLMC_OK;
}

}  // namespace

extern "C" {

mlmc_status mlmc_server_create(const mlmc_config* cfg, const mlmc_server_config* scfg, mlmc_server** out) {
  if (!cfg || !scfg || !out) return MLMC_ERR_INVALID_ARG;
  *out = nullptr;
  return start_server(std::unique_ptr<Backend>(new StripBackend(*cfg)), scfg, out);
}

mlmc_status mlmcp_server_create(const mlmcp_config* cfg, const mlmc_server_config* scfg, double mlmc_m,
                                double mlmc_alpha, mlmc_server** out) {
  if (!cfg || !scfg || !out) return MLMC_ERR_INVALID_ARG;
  *out = nullptr;
  return start_server(std::unique_ptr<Backend>(new PanelBackend(*cfg, mlmc_m, mlmc_alpha)), scfg, out);
}

mlmc_status mlmc_server_submit(mlmc_server* s, const mlmc_request* reqs, int64_t n) {
  if (!s || n < 0 || (n > 0 && !reqs)) return MLMC_ERR_INVALID_ARG;
  for (int64_t k = 0; k < n; ++k) {
    const mlmc_request& r = reqs[k];
    const int L = s->be->levels();
    const bool ok = r.level >= 0 && r.level < L &&
                    (r.kind == MLMC_REQ_SELECTIVE || (r.kind == MLMC_REQ_SOLVE && r.mesh_level >= 0 && r.mesh_level < L));
    if (!ok) {
      s->record_error("request with an invalid kind, level or mesh");
      return MLMC_ERR_INVALID_ARG;
    }
  }
  const Clock::time_point t0 = Clock::now();
  {
    std::lock_guard<std::mutex> g(s->mu);
    for (int64_t k = 0; k < n; ++k) {
      Pending p;
      p.req = reqs[k];
      p.t0 = t0;
      s->queue.push_back(p);
    }
    s->outstanding += n;
  }
  s->cv_work.notify_all();
  return MLMC_OK;
}

mlmc_status mlmc_server_poll(mlmc_server* s, mlmc_result* out, int64_t max, int64_t* count) {
  if (!s || !count || max < 0 || (max > 0 && !out)) return MLMC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  int64_t k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *count = k;
  return MLMC_OK;
}

mlmc_status mlmc_server_drain(mlmc_server* s, double timeout_ms) {
  if (!s) return MLMC_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(std::max(0.0, timeout_ms)),
                                      [&] { return s->outstanding == 0; });
  return ok ? MLMC_OK : MLMC_ERR_TIMEOUT;
}

mlmc_status mlmc_server_counters(mlmc_server* s, int64_t* batches, int64_t* solves, double* peak_bytes) {
  if (!s) return MLMC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  if (batches) *batches = s->batches;
  if (solves) *solves = s->solves;
  if (peak_bytes) *peak_bytes = s->peak;
  return MLMC_OK;
}

void mlmc_server_destroy(mlmc_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->threads) t.join();
  s->be.reset();   // the worker contexts, before their streams
  for (auto st : s->streams) cudaStreamDestroy(st);
  s->pool.release();
  delete s;
}

mlmc_status mlmc_failure_estimate(const mlmc_result* res, int64_t n, double threshold, int32_t k,
                                  int32_t two_level, double* estimate, double* mean, double* var) {
  if (n < 0 || (n > 0 && !res) || k < 0 || !estimate) return MLMC_ERR_INVALID_ARG;
  int64_t cnt[MLMC_SR_MAX_LEVELS] = {0}, plus[MLMC_SR_MAX_LEVELS] = {0}, minus[MLMC_SR_MAX_LEVELS] = {0};
  int top = -1;
  for (int64_t i = 0; i < n; ++i)
    if (res[i].status == 0 && res[i].kind == MLMC_REQ_SELECTIVE) top = std::max(top, (int)res[i].level);
  for (int64_t i = 0; i < n; ++i) {
    const mlmc_result& r = res[i];
    if (r.status != 0 || r.kind != MLMC_REQ_SELECTIVE || r.level < 0 || r.level >= MLMC_SR_MAX_LEVELS) continue;
    int y;
    if (r.level == 0) {
      y = r.q_fine;
    } else if (!two_level) {
      y = r.q_fine - r.q_coarse;
    } else if (r.level == top) {
      y = r.q_fine - r.q_mesh0;
    } else {
      continue;   // intermediate levels take no part in the two-level form
    }
    ++cnt[r.level];
    plus[r.level] += y == 1;
    minus[r.level] += y == -1;
  }
  double est = 0.0;
  for (int l = 0; l < MLMC_SR_MAX_LEVELS; ++l) {
    double e = 0.0, v = 0.0;
    if (cnt[l] > 0) {
      const double pp = (double)(plus[l] + k) / (double)(cnt[l] + k);
      const double pm = l == 0 ? 0.0 : (double)(minus[l] + k) / (double)(cnt[l] + k);
      e = pp - pm;
      v = pp + pm - e * e;
      est += e;
    }
    if (mean) mean[l] = e;
    if (var) var[l] = v;
  }
  *estimate = est;
  return MLMC_OK;
}

const char* mlmc_server_last_error(const mlmc_server* s) { return s ? s->err : g_server_error.c_str(); }

}  // extern "C"
