// Solve service over resident hierarchies (the hhg_server_* entry points of
// include/hhg.h): a FIFO queue, admission by free slot and HBM budget, a
// cache of built and fitted hierarchies keyed by geometry and level, one
// host worker thread with its own CUDA stream per slot, so that admitted
// requests overlap on the device, and optional continuous batching (queued
// requests of one key merged into one batched solve, each right-hand side
// stopped at its own convergence).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "common.h"
#include "shell.h"

namespace hhg {

namespace {

using Clock = std::chrono::steady_clock;
using Key = std::tuple<double, double, int, int, int>;

Key key_of(const hhg_problem& p) { return Key{p.r_inner, p.r_outer, p.tang_refine, p.radial_layers, p.L}; }
// The bytes of a built hierarchy depend on the macro mesh and level only.
using SizeKey = std::tuple<int, int, int>;
SizeKey size_key_of(const hhg_problem& p) { return SizeKey{p.tang_refine, p.radial_layers, p.L}; }

struct Request {
  int64_t id = 0;
  hhg_problem prob{};
  int nrhs = 0;
  int64_t n_total = 0;
  std::vector<double> f, u, relres;
  hhg_request_info info{};
  std::string error;
  bool done = false;
  bool waited = false;
};

struct Resident {
  Key key;
  hhg_shell* shell = nullptr;
  size_t bytes = 0;
  bool busy = false;
  double last_used = 0.0;
  // request vectors kept with the hierarchy (stable addresses let its
  // captured V-cycle graph be replayed by later requests)
  double* df = nullptr;
  double* du = nullptr;
  size_t vec_cap = 0;  // doubles per vector buffer
};

}  // namespace
}  // namespace hhg

using namespace hhg;

struct hhg_server {
  hhg_server_desc d{};
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::map<int64_t, std::unique_ptr<Request>> requests;
  std::vector<std::unique_ptr<Resident>> cache;  // stable addresses: workers hold pointers
  size_t used = 0;       // bytes of resident hierarchies + admitted request vectors
  bool building = false; // one hierarchy is built at a time (it may take the whole free budget)
  int64_t next_id = 1;
  int64_t n_built = 0;
  int64_t n_evicted = 0;
  std::map<hhg::SizeKey, size_t> built_bytes;  // bytes of the last hierarchy built per mesh and level
  int active = 0;
  bool stop = false;
  std::vector<std::thread> workers;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  size_t free_budget() const {
    if (d.hbm_budget_bytes == 0) return (size_t)-1;
    return d.hbm_budget_bytes > used ? d.hbm_budget_bytes - used : 0;
  }
};

namespace {

int64_t free_nodes_of(const hhg_problem& p, int64_t* n_total) {
  // (N_r + 1) spherical layers of 10 n_t^2 + 2 nodes; the two boundary
  // layers are Dirichlet
  const int64_t N = (int64_t)1 << p.L;
  const int64_t nt = N << p.tang_refine, nr = N * p.radial_layers;
  const int64_t layer = 10 * nt * nt + 2;
  *n_total = (nr + 1) * layer;
  return (nr - 1) * layer;
}

size_t vec_bytes_of(const Request* r) { return (size_t)2 * r->nrhs * r->n_total * sizeof(double); }

// Continuous batching: the requests queued for the same key as the picked
// one join its solve, in arrival order, while the right-hand sides fit
// max_batch_rhs and their vectors the budget.
void join_same_key(hhg_server* s, std::vector<Request*>* grp) {
  if (s->d.max_batch_rhs <= 1) return;
  const Key k = key_of((*grp)[0]->prob);
  int rhs = (*grp)[0]->nrhs;
  size_t bytes = vec_bytes_of((*grp)[0]);
  for (auto it = s->pending.begin(); it != s->pending.end();) {
    Request* r = *it;
    if (key_of(r->prob) == k && rhs + r->nrhs <= s->d.max_batch_rhs && bytes + vec_bytes_of(r) <= s->free_budget()) {
      grp->push_back(r);
      rhs += r->nrhs;
      bytes += vec_bytes_of(r);
      it = s->pending.erase(it);
    } else {
      ++it;
    }
  }
}

// Picks the next admissible request under the lock: the first queued one
// whose hierarchy is resident and idle, or for which a new hierarchy may be
// built now, together with the queued requests that join it.  Returns the
// group and the cache slot (-1 = build).
bool pick(hhg_server* s, std::vector<Request*>* grp, int* slot) {
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
    Request* r = *it;
    if (vec_bytes_of(r) > s->free_budget()) continue;
    const Key k = key_of(r->prob);
    int idle = -1;
    bool exists = false;
    for (size_t c = 0; c < s->cache.size(); ++c)
      if (s->cache[c]->key == k) {
        exists = true;
        if (!s->cache[c]->busy) idle = (int)c;
      }
    // while a hierarchy is being built, and (with continuous batching) while
    // the key's hierarchy is busy, wait for it rather than build a copy
    if (idle < 0 && (s->building || (exists && s->d.max_batch_rhs > 1))) continue;
    grp->assign(1, r);
    *slot = idle;
    s->pending.erase(it);
    join_same_key(s, grp);
    return true;
  }
  return false;
}

// Evicts idle hierarchies, least recently used first, until `need` bytes
// are free (or nothing idle is left).
void evict_for(hhg_server* s, size_t need) {
  while (s->free_budget() < need) {
    int lru = -1;
    for (size_t c = 0; c < s->cache.size(); ++c)
      if (!s->cache[c]->busy && (lru < 0 || s->cache[c]->last_used < s->cache[lru]->last_used)) lru = (int)c;
    if (lru < 0) return;
    cudaDeviceSynchronize();
    cudaFree(s->cache[lru]->df);
    cudaFree(s->cache[lru]->du);
    hhg_destroy(s->cache[lru]->shell);
    s->used -= s->cache[lru]->bytes;
    s->cache.erase(s->cache.begin() + lru);
    ++s->n_evicted;
  }
}

// Solves a group of requests of one key as one batched V-cycle solve on the
// resident hierarchy: right-hand sides in group order.  With continuous
// batching each right-hand side is stopped on its own (hhg_shell::
// freeze_host), so every request gets the iterate and relative residual of
// the cycle where it met the tolerance.
void run_group(hhg_server* s, const std::vector<Request*>& grp, Resident& res, cudaStream_t st) {
  const int64_t nt = grp[0]->n_total;
  int T = 0;
  for (const Request* r : grp) T += r->nrhs;
  const size_t n = (size_t)T * nt;
  hhg_shell* sh = res.shell;
  hhg_status status = HHG_OK;
  std::string error;
  if (n > res.vec_cap) {
    if (res.df) cudaFreeAsync(res.df, st);
    if (res.du) cudaFreeAsync(res.du, st);
    res.df = res.du = nullptr;
    res.vec_cap = 0;
    if (cudaMallocAsync((void**)&res.df, n * sizeof(double), st) != cudaSuccess ||
        cudaMallocAsync((void**)&res.du, n * sizeof(double), st) != cudaSuccess) {
      cudaGetLastError();
      if (res.df) cudaFreeAsync(res.df, st);
      res.df = res.du = nullptr;
    } else {
      res.vec_cap = n;
    }
  }
  double* df = res.df;
  double* du = res.du;
  const bool merge = s->d.max_batch_rhs > 1;
  std::vector<double> rel((size_t)T, 0.0), uh;
  std::vector<int> fc((size_t)T, 0);
  int cycles = 0;
  if (!df || !du) {
    status = HHG_ENOMEM;
    error = "request vectors do not fit on the device";
  } else {
    size_t o = 0;
    for (const Request* r : grp) {
      cudaMemcpyAsync(df + o, r->f.data(), r->f.size() * sizeof(double), cudaMemcpyHostToDevice, st);
      o += r->f.size();
    }
    cudaMemsetAsync(du, 0, n * sizeof(double), st);
    if (merge) {
      uh.resize(n);
      sh->freeze_host = uh.data();
      sh->freeze_cycle = fc.data();
    }
    status = hhg_vcycle(sh, HHG_OP_LSQP, s->d.dtype, df, du, s->d.nu1, s->d.nu2, s->d.max_cycles, s->d.rtol, T,
                        rel.data(), &cycles, st);
    sh->freeze_host = nullptr;
    sh->freeze_cycle = nullptr;
    if (status != HHG_OK) error = hhg_last_error();
    if (!merge && cudaMemcpyAsync(grp[0]->u.data(), du, n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess &&
        status == HHG_OK) {
      status = HHG_ECUDA;
      error = "copy of the solution failed";
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && status == HHG_OK) {
    status = HHG_ECUDA;
    error = "stream failed";
  }
  size_t o = 0;
  int b0 = 0;
  for (Request* r : grp) {
    hhg_status rs = status;
    int rc = cycles;
    bool conv = true;
    if (merge) {
      rc = 0;
      for (int b = 0; b < r->nrhs; ++b) rc = std::max(rc, fc[(size_t)b0 + b]);
      if (!uh.empty()) std::memcpy(r->u.data(), uh.data() + o, r->u.size() * sizeof(double));
    }
    for (int b = 0; b < r->nrhs; ++b) {
      r->relres[(size_t)b] = rel[(size_t)b0 + b];
      conv = conv && rel[(size_t)b0 + b] <= s->d.rtol;
    }
    // a merged solve that did not converge fails only the requests whose
    // own right-hand sides missed the tolerance
    if (rs == HHG_ENOCONV && conv) rs = HHG_OK;
    r->info.status = rs;
    r->info.cycles = rc;
    r->info.batch_rhs = T;
    r->error = rs == HHG_OK ? std::string() : error;
    o += r->u.size();
    b0 += r->nrhs;
  }
}

void worker(hhg_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    std::vector<Request*> grp;
    int slot = -1;
    size_t vec_bytes = 0;
    hhg_shell* sh_cached = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return (s->stop && s->pending.empty()) || pick(s, &grp, &slot); });
      if (grp.empty()) break;
      for (const Request* q : grp) vec_bytes += vec_bytes_of(q);
      s->used += vec_bytes;
      ++s->active;
      if (slot >= 0) {
        s->cache[slot]->busy = true;
        sh_cached = s->cache[slot]->shell;
      } else {
        s->building = true;
      }
      const double t = s->now();
      for (Request* q : grp) {
        q->info.reused = slot >= 0 ? 1 : 0;
        q->info.t_start = t;
      }
    }
    Request* r = grp[0];
    hhg_shell* sh = nullptr;
    if (slot >= 0) {
      sh = sh_cached;
    } else {
      // build and fit a new hierarchy within the budget left (evicting idle
      // ones when it does not fit)
      hhg_status st_build = HHG_ENOMEM;
      std::string err;
      for (int attempt = 0; attempt < 2 && st_build == HHG_ENOMEM; ++attempt) {
        size_t budget;
        {
          std::lock_guard<std::mutex> lk(s->mu);
          // evict least-recently-used idle hierarchies: as many as the bytes
          // of an earlier build of this mesh and level need, else all idle ones
          if (attempt == 1) {
            auto h = s->built_bytes.find(size_key_of(r->prob));
            evict_for(s, h != s->built_bytes.end() ? h->second : s->d.hbm_budget_bytes);
          }
          budget = s->d.hbm_budget_bytes ? s->free_budget() : 0;
        }
        if (s->d.hbm_budget_bytes && budget == 0) continue;
        hhg_shell_desc sd{r->prob.r_inner, r->prob.r_outer, r->prob.tang_refine, r->prob.radial_layers, r->prob.L,
                          budget};
        st_build = hhg_setup_shell(&sd, st, &sh);
        if (st_build == HHG_OK) {
          // admitted: later growth (FP32 buffers, more right-hand sides) is
          // accounted after each request rather than refused
          sh->alloc.budget = 0;
          st_build = hhg_fit_surrogate(sh, s->d.q, s->d.j, st);
          if (st_build != HHG_OK) {
            err = hhg_last_error();
            hhg_destroy(sh);
            sh = nullptr;
          }
        } else {
          err = hhg_last_error();
        }
      }
      std::lock_guard<std::mutex> lk(s->mu);
      s->building = false;
      s->cv_work.notify_all();
      if (!sh) {
        for (Request* q : grp) {
          q->info.status = st_build;
          q->error = err;
        }
      } else {
        auto res = std::make_unique<Resident>();
        res->key = key_of(r->prob);
        res->shell = sh;
        res->bytes = sh->alloc.used;
        res->busy = true;
        s->built_bytes[size_key_of(r->prob)] = res->bytes;
        s->used += res->bytes;
        s->cache.push_back(std::move(res));
        ++s->n_built;
      }
    }
    if (sh) {
      Resident* res = nullptr;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& c : s->cache)
          if (c->shell == sh) res = c.get();
      }
      run_group(s, grp, *res, st);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const double t = s->now();
      for (Request* q : grp) {
        q->info.t_end = t;
        q->done = true;
      }
      s->used -= vec_bytes;
      --s->active;
      for (auto& c : s->cache)
        if (c->shell == sh) {
          c->busy = false;
          c->last_used = t;
          // a hierarchy may have grown (FP32 buffers, batch capacity)
          s->used += sh->alloc.used - c->bytes;
          c->bytes = sh->alloc.used;
        }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

hhg_status hhg_problem_nodes(const hhg_problem* p, int64_t* n_total, int64_t* n_free) {
  if (!p || p->L < 2 || p->L > 10 || p->tang_refine < 0 || p->radial_layers < 1) {
    set_error("invalid problem");
    return HHG_EINVAL;
  }
  int64_t nt = 0;
  const int64_t nf = free_nodes_of(*p, &nt);
  if (n_total) *n_total = nt;
  if (n_free) *n_free = nf;
  set_error("");
  return HHG_OK;
}

hhg_status hhg_server_create(const hhg_server_desc* d, hhg_server** out) {
  if (!d || !out || d->max_inflight < 1 || d->max_inflight > 64 || d->q < 1 || d->q > 3 || d->j < 1 ||
      d->rtol < 0 || d->max_cycles < 1 || (d->dtype != HHG_F64 && d->dtype != HHG_F32) || d->max_batch_rhs < 0) {
    set_error("invalid server descriptor");
    return HHG_EINVAL;
  }
  hhg_server* s = new hhg_server();
  s->d = *d;
  s->t0 = Clock::now();
  cudaGetDevice(&s->device);
  for (int w = 0; w < d->max_inflight; ++w) s->workers.emplace_back(worker, s);
  *out = s;
  set_error("");
  return HHG_OK;
}

hhg_status hhg_server_submit(hhg_server* s, const hhg_problem* p, const double* f, int nrhs, int64_t* ticket) {
  if (!s || !p || !f || nrhs < 1 || !ticket) {
    set_error("invalid submit argument");
    return HHG_EINVAL;
  }
  int64_t nt = 0;
  if (hhg_problem_nodes(p, &nt, nullptr) != HHG_OK) return HHG_EINVAL;
  if (!(p->r_inner > 0 && p->r_outer > p->r_inner)) {
    set_error("need 0 < r_inner < r_outer");
    return HHG_EINVAL;
  }
  auto r = std::make_unique<Request>();
  r->prob = *p;
  r->nrhs = nrhs;
  r->n_total = nt;
  r->f.assign(f, f + (size_t)nrhs * nt);
  r->u.assign((size_t)nrhs * nt, 0.0);
  r->relres.assign((size_t)nrhs, 0.0);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->info.t_submit = s->now();
    *ticket = r->id;
    s->pending.push_back(r.get());
    s->requests[r->id] = std::move(r);
  }
  s->cv_work.notify_all();
  set_error("");
  return HHG_OK;
}

hhg_status hhg_server_wait(hhg_server* s, int64_t ticket, double* u, double* relres, hhg_request_info* info) {
  if (!s) {
    set_error("NULL server");
    return HHG_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end() || it->second->waited) {
    set_error("unknown ticket");
    return HHG_EINVAL;
  }
  Request* r = it->second.get();
  s->cv_done.wait(lk, [&] { return r->done; });
  r->waited = true;
  if (u) std::memcpy(u, r->u.data(), r->u.size() * sizeof(double));
  if (relres) std::memcpy(relres, r->relres.data(), r->relres.size() * sizeof(double));
  if (info) *info = r->info;
  const hhg_status st = r->info.status;
  set_error(r->error);
  s->requests.erase(it);
  return st;
}

hhg_status hhg_server_stats(hhg_server* s, int* n_resident, size_t* bytes, int64_t* n_built, int64_t* n_evicted) {
  if (!s) {
    set_error("NULL server");
    return HHG_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  size_t b = 0;
  for (auto& c : s->cache) b += c->bytes;
  if (n_resident) *n_resident = (int)s->cache.size();
  if (bytes) *bytes = b;
  if (n_built) *n_built = s->n_built;
  if (n_evicted) *n_evicted = s->n_evicted;
  set_error("");
  return HHG_OK;
}

hhg_status hhg_server_destroy(hhg_server* s) {
  if (!s) return HHG_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  cudaDeviceSynchronize();
  for (auto& c : s->cache) {
    cudaFree(c->df);
    cudaFree(c->du);
    hhg_destroy(c->shell);
  }
  delete s;
  set_error("");
  return HHG_OK;
}

}  // extern "C"
