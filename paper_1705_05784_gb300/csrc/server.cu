// Request server: continuous batching of independent pressure solves, and
// time-step updates against resident setups.
//
// Callers submit problems (copied at submission) and collect results by
// ticket.  Worker threads, each with its own CUDA stream, take whatever has
// arrived -- up to max_batch new realisations of the oldest request's kind (a
// wide coarse band to factor, or not), no more than the device-memory budget
// allows next to the micro-batches in flight and the resident setups -- set
// the micro-batch up, solve it and reconstruct its fluxes, while the other
// workers do the same with the requests that arrived in the meantime.  A
// request's result does not depend on what it was batched with (one CTA per
// instance in the solve, fixed reduction orders), up to the rounding of the
// coarse operator's atomic sums.
//
// A micro-batch's context stays resident after it completes (coarse grids,
// P, the coarse factors, ILU(0)).  A time-step update request names an
// earlier request (its base) and a mobility scale per cell: a worker applies
// fams_update_batch to the base's resident context (basis functions kept,
// Sec. 3.1 end), solves only the updated instances (fams_solve_subset) from
// the base's pressure, and reconstructs their fluxes.  The least recently
// used idle setups are destroyed when a micro-batch needs their memory; an
// update of an evicted base sets the base problem up again first.  The paper
// has no counterpart: this is the deployment layer around its solver.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace fams {
void set_error(const std::string& msg);
}

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

bool on_device(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// a result vector into a caller array (host or device memory)
int copy_out(double* dst, const std::vector<double>& src) {
  if (src.empty()) return FAMS_OK;
  if (on_device(dst)) {
    cudaError_t e = cudaMemcpy(dst, src.data(), sizeof(double) * src.size(), cudaMemcpyDefault);
    if (e != cudaSuccess) {
      fams::set_error(std::string("copying a result: ") + cudaGetErrorString(e));
      return FAMS_ECUDA;
    }
  } else {
    std::memcpy(dst, src.data(), sizeof(double) * src.size());
  }
  return FAMS_OK;
}

// a caller array of n doubles (host or device memory) into a host vector
int copy_in(std::vector<double>& dst, const double* src, size_t n) {
  dst.resize(n);
  if (n == 0) return FAMS_OK;
  if (on_device(src)) {
    cudaError_t e = cudaMemcpy(dst.data(), src, sizeof(double) * n, cudaMemcpyDefault);
    if (e != cudaSuccess) {
      fams::set_error(std::string("copying a request's array: ") + cudaGetErrorString(e));
      return FAMS_ECUDA;
    }
  } else {
    std::memcpy(dst.data(), src, sizeof(double) * n);
  }
  return FAMS_OK;
}

struct Resident;

struct Request {
  long long id = 0;
  fams_grid grid{};
  std::vector<double> perm, xy, kf, rhs;
  fams_fracs fr{};
  fams_opts opts{};
  size_t mem = 0;
  bool heavy = false;   // large coarse factorisation: batched only with its own kind
  // time-step update of request `base`: mobility scale per cell; x0 is the
  // base's pressure, copied when the update is taken
  bool update = false;
  long long base = 0;
  std::vector<double> scale, x0;
  // a new realisation that succeeded: its resident context and instance there
  Resident* res = nullptr;
  int inst = -1;
  bool solo = false;    // solved again alone: its instance in the micro-batch context failed
  // results
  std::vector<double> x, face, nnc;
  fams_stats st{};
  int status = FAMS_OK;
  std::string err;   // detail of a failure
  bool done = false;
  double t_submit = 0, t_start = 0, t_done = 0;
};

// a finished micro-batch's context, kept for time-step updates of its members
struct Resident {
  fams_ctx* ctx = nullptr;
  size_t mem = 0;
  std::vector<long long> members;   // tickets of its instances, by instance
  int alive = 0;                    // members not yet released
  bool busy = false;                // a worker runs an update on it
  double last_use = 0;
};

// device bytes of one instance, estimated from its size: fine system, P,
// ILU(0) (plain and level-ordered), work and Krylov vectors per unknown, the
// dense coarse operators (R^FE and R^FV) per coarse unknown squared
size_t estimate_bytes(const Request& r) {
  long long cells = (long long)r.grid.nx * r.grid.ny * (r.grid.dim == 3 ? r.grid.nz : 1);
  long long cr = (long long)std::max(1, r.opts.coarsen[0]) * std::max(1, r.opts.coarsen[1]) *
                 (r.grid.dim == 3 ? std::max(1, r.opts.coarsen[2]) : 1);
  long long nfc = 0;
  for (int f = 0; f < r.fr.n; ++f) {
    const double* s = &r.xy[(size_t)f * (r.grid.dim == 3 ? 6 : 4)];
    double L = sqrt((s[2] - s[0]) * (s[2] - s[0]) + (s[3] - s[1]) * (s[3] - s[1]));
    nfc += (long long)(L / std::max(r.fr.h_f, 1e-9) + 1) * (r.grid.dim == 3 ? r.grid.nz : 1);
  }
  long long n = cells + nfc;
  long long nc = cells / cr + nfc / std::max(1, r.opts.frac_dmin > 0 ? r.opts.frac_dmin : 8) + 8;
  long long kry = r.opts.krylov == FAMS_KRYLOV_GMRES ? (long long)(r.opts.restart + 1) * 8 : 0;
  return (size_t)(n * (1200 + kry) + nc * nc * 16);
}

// work of the coarse band factorisation, nc kl^2 with kl about three planes
// (3D) or three lines (2D) of coarse nodes.  A heavy request runs alone on
// the whole GPU (fams_opts.grid_solve = 1 unless the caller chose -1): its
// band factorisation on one SM would take seconds and hold the micro-batch
// and the SMs of the small requests beside it.
bool estimate_heavy(const Request& r) {
  auto nodes = [](int n, int c) { return (double)std::max(1, (n + std::max(1, c) - 1) / std::max(1, c)); };
  double cx = nodes(r.grid.nx, r.opts.coarsen[0]), cy = nodes(r.grid.ny, r.opts.coarsen[1]);
  double cz = r.grid.dim == 3 ? nodes(r.grid.nz, r.opts.coarsen[2]) : 1.0;
  double nc = cx * cy * cz;
  double kl = 3.0 * (r.grid.dim == 3 ? cx * cy : cx);
  return nc * kl * kl > 2e7;
}

}  // namespace

struct fams_server {
  int device = 0;
  fams_server_opts o{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::unordered_map<long long, Request*> all;
  long long next_id = 1;
  size_t inflight = 0;
  std::vector<Resident*> residents;
  size_t resident_mem = 0;
  bool stop = false;
  std::vector<std::thread> workers;
};

namespace {

Request* find(fams_server* s, long long ticket) {
  auto it = s->all.find(ticket);
  return it == s->all.end() ? nullptr : it->second;
}

// the problems of a micro-batch as fams_setup_batch takes them (pointers into
// the requests)
struct Inputs {
  std::vector<fams_grid> grids;
  std::vector<const double*> perms;
  std::vector<fams_fracs> fracs;
  std::vector<fams_opts> opts;
  explicit Inputs(const std::vector<Request*>& batch, bool with_flux) {
    const size_t n = batch.size();
    grids.resize(n); perms.resize(n); fracs.resize(n); opts.resize(n);
    for (size_t i = 0; i < n; ++i) {
      grids[i] = batch[i]->grid;
      perms[i] = batch[i]->perm.data();
      fracs[i] = batch[i]->fr;
      fracs[i].xy = batch[i]->xy.empty() ? nullptr : batch[i]->xy.data();
      fracs[i].kf = batch[i]->kf.empty() ? nullptr : batch[i]->kf.data();
      opts[i] = batch[i]->opts;
      opts[i].prepare_flux = with_flux ? 1 : 0;
    }
  }
};

// solve the listed instances of ctx (request k on instance list[k], from the
// initial guess in its x) and reconstruct their fluxes; statuses per request
void solve_and_flux(fams_server* s, fams_ctx* ctx, const std::vector<int>& list,
                    std::vector<Request*>& reqs) {
  const int n = (int)reqs.size();
  std::vector<const double*> rhs(n);
  std::vector<double*> xs(n);
  for (int k = 0; k < n; ++k) {
    Request* r = reqs[k];
    int nm = 0, nf = 0, nfaces = 0, nnnc = 0;
    fams_sizes(ctx, list[k], &nm, &nf, nullptr, &nfaces, &nnnc);
    if (r->x.size() != (size_t)nm + nf) r->x.assign((size_t)nm + nf, 0.0);
    if (!r->rhs.empty() && r->rhs.size() != r->x.size()) r->rhs.resize(r->x.size(), 0.0);
    rhs[k] = r->rhs.empty() ? nullptr : r->rhs.data();
    xs[k] = r->x.data();
    if (s->o.with_flux) {
      r->face.assign((size_t)nfaces, 0.0);
      r->nnc.assign((size_t)std::max(nnnc, 1), 0.0);
    }
  }
  std::vector<fams_stats> stats(n);
  int ss = fams_solve_subset(ctx, n, list.data(), rhs.data(), xs.data(), s->o.tol, stats.data());
  std::string serr = ss == FAMS_OK ? "" : fams_last_error();
  std::vector<int> fst(n, FAMS_OK);
  if (s->o.with_flux && ss != FAMS_ECUDA && ss != FAMS_EINVAL) {
    if (n == fams_num_instances(ctx)) {   // list = 0..n-1: one reconstruction for all
      std::vector<double*> fs(n), ns(n);
      for (int k = 0; k < n; ++k) {
        fs[k] = reqs[k]->face.data();
        ns[k] = reqs[k]->nnc.data();
      }
      fams_flux_batch(ctx, xs.data(), fs.data(), ns.data(), fst.data());
    } else {
      for (int k = 0; k < n; ++k)
        if (stats[k].converged)
          fst[k] = fams_flux(ctx, list[k], xs[k], reqs[k]->face.data(), reqs[k]->nnc.data());
    }
  }
  for (int k = 0; k < n; ++k) {
    Request* r = reqs[k];
    r->st = stats[k];
    if (ss == FAMS_ECUDA || ss == FAMS_EINVAL || ss == FAMS_ETIMEOUT) r->status = ss;
    else if (!stats[k].converged) r->status = std::isfinite(stats[k].rel_residual) ? FAMS_ENOCONV
                                                                                  : FAMS_EBREAKDOWN;
    else r->status = fst[k];
    if (r->status != FAMS_OK) r->err = r->status == fst[k] ? "flux reconstruction failed" : serr;
  }
}

// set up, solve and reconstruct one micro-batch of new realisations; on a
// setup failure each request is retried alone so that one bad problem fails
// only itself.  Returns the context (to keep resident) or null.
fams_ctx* run_batch(fams_server* s, std::vector<Request*>& batch) {
  const int n = (int)batch.size();
  Inputs in(batch, s->o.with_flux != 0);
  for (Request* r : batch) r->t_start = now_ms();
  fams_ctx* ctx = nullptr;
  int st = fams_setup_batch(n, in.grids.data(), in.perms.data(), in.fracs.data(), in.opts.data(),
                            &ctx);
  if (st != FAMS_OK) {
    if (n > 1) {
      for (Request* r : batch) {
        std::vector<Request*> one{r};
        fams_ctx* c = run_batch(s, one);
        if (c) fams_destroy(c);   // (a retried request is not kept resident)
      }
    } else {
      batch[0]->status = st;
      batch[0]->err = fams_last_error();
    }
    return nullptr;
  }
  std::vector<int> list(n);
  for (int i = 0; i < n; ++i) list[i] = i;
  solve_and_flux(s, ctx, list, batch);
  // a coarse system beyond the one-CTA path's limits (a band wider than its
  // shared-memory chunks) fails the batch's solve: such requests run again
  // alone on the whole GPU (not kept resident: their updates set them up again)
  if (n > 1 || batch[0]->opts.grid_solve != 1) {
    for (Request* r : batch)
      if (r->status == FAMS_ECAPACITY && r->opts.grid_solve != -1) {
        r->opts.grid_solve = 1;
        r->solo = true;
        r->status = FAMS_OK;
        r->err.clear();
        std::vector<Request*> one{r};
        fams_ctx* c = run_batch(s, one);
        if (c) fams_destroy(c);
      }
  }
  return ctx;
}

// time-step updates on a resident context: each request's base is instance
// list[k]; the other instances go back to their setup operators
void run_update(fams_server* s, Resident* R, std::vector<Request*>& batch,
                const std::vector<int>& list) {
  const int B = fams_num_instances(R->ctx);
  std::vector<const double*> scales(B, nullptr);
  for (size_t k = 0; k < batch.size(); ++k) {
    scales[list[k]] = batch[k]->scale.data();
    batch[k]->t_start = now_ms();
    batch[k]->x = batch[k]->x0;
  }
  int st = fams_update_batch(R->ctx, scales.data());
  if (st != FAMS_OK) {
    for (Request* r : batch) {
      r->status = st;
      r->err = fams_last_error();
    }
    return;
  }
  solve_and_flux(s, R->ctx, list, batch);
}

// time-step updates whose base is no longer resident: the base problems are
// set up again (the update requests carry copies of them), then updated
void run_update_fresh(fams_server* s, std::vector<Request*>& batch) {
  const int n = (int)batch.size();
  Inputs in(batch, s->o.with_flux != 0);
  for (Request* r : batch) {
    r->t_start = now_ms();
    r->x = r->x0;
  }
  fams_ctx* ctx = nullptr;
  int st = fams_setup_batch(n, in.grids.data(), in.perms.data(), in.fracs.data(), in.opts.data(),
                            &ctx);
  if (st == FAMS_OK) {
    std::vector<const double*> scales(n);
    for (int i = 0; i < n; ++i) scales[i] = batch[i]->scale.data();
    st = fams_update_batch(ctx, scales.data());
  }
  if (st != FAMS_OK) {
    for (Request* r : batch) {
      r->status = st;
      r->err = fams_last_error();
    }
    if (ctx) fams_destroy(ctx);
    return;
  }
  std::vector<int> list(n);
  for (int i = 0; i < n; ++i) list[i] = i;
  solve_and_flux(s, ctx, list, batch);
  fams_destroy(ctx);
}

// destroys resident contexts (outside the server lock)
void destroy_all(std::vector<fams_ctx*>& dead) {
  for (fams_ctx* c : dead) fams_destroy(c);
  dead.clear();
}

// takes a resident context out of the server's list (caller holds the lock);
// its members fall back to a fresh setup for later updates
fams_ctx* retire(fams_server* s, Resident* R) {
  for (long long t : R->members) {
    Request* m = find(s, t);
    if (m && m->res == R) m->res = nullptr;
  }
  s->residents.erase(std::find(s->residents.begin(), s->residents.end(), R));
  s->resident_mem -= R->mem;
  fams_ctx* c = R->ctx;
  delete R;
  return c;
}

// frees room for `need` bytes by retiring the least recently used idle
// resident contexts (caller holds the lock); true if it fits afterwards
bool make_room(fams_server* s, size_t need, std::vector<fams_ctx*>& dead) {
  while (s->inflight + s->resident_mem + need > (size_t)s->o.hbm_budget) {
    Resident* lru = nullptr;
    for (Resident* R : s->residents)
      if (!R->busy && (!lru || R->last_use < lru->last_use)) lru = R;
    if (!lru) return false;
    dead.push_back(retire(s, lru));
  }
  return true;
}

// the next micro-batch (caller holds the lock): a time-step update batch
// (every pending update of one resident context, distinct bases) or a batch
// of new realisations of the oldest one's kind.  Updates whose base failed or
// was released fail here (`finished`).  kind: 0 none, 1 new, 2 update on R,
// 3 update on a fresh setup.
int pick(fams_server* s, std::vector<Request*>& batch, size_t& mem, Resident*& R,
         std::vector<int>& list, std::vector<Request*>& finished, std::vector<fams_ctx*>& dead) {
  bool new_waits = false;   // the oldest new realisation waits for memory: so do later ones
  for (auto it = s->pending.begin(); it != s->pending.end();) {
    Request* r = *it;
    if (!r->update) {
      // new realisations: the oldest runnable one and later ones of its kind
      const bool kind = r->heavy;
      const bool idle = s->inflight == 0;
      if (new_waits || (!make_room(s, r->mem, dead) && !idle)) {
        new_waits = true;
        ++it;
        continue;
      }
      const int cap = kind ? 1 : s->o.max_batch;   // a heavy request runs alone
      for (auto jt = it; jt != s->pending.end() && (int)batch.size() < cap;) {
        Request* q = *jt;
        if (q->update || q->heavy != kind) { ++jt; continue; }
        if (!batch.empty() && !make_room(s, mem + q->mem, dead)) break;
        batch.push_back(q);
        mem += q->mem;
        jt = s->pending.erase(jt);
      }
      return 1;
    }
    Request* b = find(s, r->base);
    if (!b || (b->done && b->status != FAMS_OK) || (b->done && b->update)) {
      r->status = FAMS_EINVAL;
      r->err = !b ? "base request released" : b->update ? "base request is itself an update"
                                                       : "base request failed";
      finished.push_back(r);
      it = s->pending.erase(it);
      continue;
    }
    if (!b->done || (b->res && b->res->busy)) { ++it; continue; }
    if (r->scale.size() != b->x.size()) {
      r->status = FAMS_EINVAL;
      r->err = "mobility scale has " + std::to_string(r->scale.size()) + " values, the base " +
               std::to_string(b->x.size()) + " unknowns";
      finished.push_back(r);
      it = s->pending.erase(it);
      continue;
    }
    if (b->res) {
      // every pending update of this resident context, one per base instance
      R = b->res;
      R->busy = true;
      for (auto jt = it; jt != s->pending.end() && (int)batch.size() < s->o.max_batch;) {
        Request* q = *jt;
        Request* qb = q->update ? find(s, q->base) : nullptr;
        if (!qb || !qb->done || qb->res != R || q->scale.size() != qb->x.size() ||
            std::find(list.begin(), list.end(), qb->inst) != list.end()) {
          ++jt;
          continue;
        }
        q->x0 = qb->x;
        batch.push_back(q);
        list.push_back(qb->inst);
        jt = s->pending.erase(jt);
      }
      return 2;
    }
    // evicted base: set it up again with the update (copies of its inputs)
    if (!make_room(s, b->mem, dead) && s->inflight != 0) { ++it; continue; }
    r->grid = b->grid; r->perm = b->perm; r->xy = b->xy; r->kf = b->kf; r->fr = b->fr;
    r->opts = b->opts;
    if (r->rhs.empty()) r->rhs = b->rhs;
    r->x0 = b->x;
    r->mem = b->mem;
    batch.push_back(r);
    mem = r->mem;
    s->pending.erase(it);
    return 3;
  }
  return 0;
}

void worker(fams_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request*> batch, finished;
    std::vector<int> list;
    std::vector<fams_ctx*> dead;
    size_t mem = 0;
    Resident* R = nullptr;
    int kind = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        if (s->stop && s->pending.empty()) return true;
        kind = pick(s, batch, mem, R, list, finished, dead);
        return kind != 0 || !finished.empty() || !dead.empty();
      });
      if (kind == 0 && finished.empty() && dead.empty() && s->stop) return;
      s->inflight += mem;
      double t = now_ms();
      for (Request* r : finished) {
        r->t_start = r->t_done = t;
        r->done = true;
      }
    }
    destroy_all(dead);
    if (!finished.empty()) s->cv_done.notify_all();
    if (kind == 0) continue;
    fams_ctx* keep = nullptr;
    if (kind == 1) keep = run_batch(s, batch);
    else if (kind == 2) run_update(s, R, batch, list);
    else run_update_fresh(s, batch);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->inflight -= mem;
      double t = now_ms();
      if (keep) {
        // resident for time-step updates of its members
        auto* K = new Resident();
        K->ctx = keep;
        K->mem = mem;
        K->last_use = t;
        for (size_t i = 0; i < batch.size(); ++i) {
          K->members.push_back(batch[i]->id);
          if (batch[i]->status == FAMS_OK && !batch[i]->solo) {
            batch[i]->res = K;
            batch[i]->inst = (int)i;
          }
        }
        K->alive = (int)batch.size();
        s->residents.push_back(K);
        s->resident_mem += mem;
      }
      if (R) {
        R->busy = false;
        R->last_use = t;
        if (R->alive == 0) dead.push_back(retire(s, R));
      }
      for (Request* r : batch) {
        r->t_done = t;
        r->done = true;
      }
    }
    destroy_all(dead);
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

using fams::set_error;

extern "C" {

int fams_server_create(const fams_server_opts* o, fams_server** out) {
  if (!o || !out) { set_error("null argument"); return FAMS_EINVAL; }
  if (o->max_batch < 1 || o->pipelines < 1 || o->pipelines > 16 || o->hbm_budget <= 0 ||
      !(o->tol >= 0.0)) {
    set_error("server options: max_batch >= 1, pipelines 1..16, hbm_budget > 0, tol >= 0");
    return FAMS_EINVAL;
  }
  fams_server* s = new fams_server();
  s->o = *o;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    set_error("no CUDA device");
    return FAMS_ECUDA;
  }
  for (int i = 0; i < o->pipelines; ++i) s->workers.emplace_back(worker, s);
  *out = s;
  return FAMS_OK;
}

int fams_server_submit(fams_server* s, const fams_grid* grid, const double* perm,
                       const fams_fracs* fracs, const fams_opts* opts, const double* rhs,
                       long long* ticket) {
  if (!s || !grid || !perm || !opts || !ticket) { set_error("null argument"); return FAMS_EINVAL; }
  if (grid->nx < 1 || grid->ny < 1 || (grid->dim == 3 && grid->nz < 1)) {
    set_error("grid sizes must be >= 1");
    return FAMS_EINVAL;
  }
  auto* r = new Request();
  r->grid = *grid;
  long long cells = (long long)grid->nx * grid->ny * (grid->dim == 3 ? grid->nz : 1);
  int cs = copy_in(r->perm, perm, (size_t)cells);
  if (cs != FAMS_OK) {
    delete r;
    return cs;
  }
  int nf = fracs ? fracs->n : 0;
  if (nf > 0) {
    if (!fracs->xy || !fracs->kf) {
      delete r;
      set_error("fracture arrays missing");
      return FAMS_EINVAL;
    }
    int w = grid->dim == 3 ? 6 : 4;
    cs = copy_in(r->xy, fracs->xy, (size_t)nf * w);
    if (cs == FAMS_OK) cs = copy_in(r->kf, fracs->kf, (size_t)nf);
    if (cs != FAMS_OK) {
      delete r;
      return cs;
    }
  }
  if (fracs) r->fr = *fracs;
  r->fr.n = nf;
  r->fr.xy = nullptr;
  r->fr.kf = nullptr;
  if (nf == 0) { r->fr.aperture = 1.0; r->fr.h_f = 1.0; }
  r->opts = *opts;
  // matrix sources; fracture sources default to 0
  if (rhs && (cs = copy_in(r->rhs, rhs, (size_t)cells)) != FAMS_OK) {
    delete r;
    return cs;
  }
  r->mem = estimate_bytes(*r);
  r->heavy = estimate_heavy(*r);
  if (r->heavy && r->opts.grid_solve == 0) r->opts.grid_solve = 1;
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      set_error("server is shutting down");
      return FAMS_EINVAL;
    }
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->pending.push_back(r);
    *ticket = r->id;
  }
  s->cv_work.notify_one();
  return FAMS_OK;
}

int fams_server_submit_update(fams_server* s, long long base, const double* mobility_scale,
                              long long n_scale, const double* rhs, long long n_rhs,
                              long long* ticket) {
  if (!s || !mobility_scale || n_scale < 0 || !ticket || (rhs && n_rhs < 0)) {
    set_error("null argument");
    return FAMS_EINVAL;
  }
  auto* r = new Request();
  r->update = true;
  r->base = base;
  int cs = copy_in(r->scale, mobility_scale, (size_t)n_scale);
  if (cs == FAMS_OK && rhs) cs = copy_in(r->rhs, rhs, (size_t)n_rhs);
  if (cs != FAMS_OK) {
    delete r;
    return cs;
  }
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      set_error("server is shutting down");
      return FAMS_EINVAL;
    }
    Request* b = find(s, base);
    if (!b || b->update) {
      delete r;
      set_error(!b ? "unknown base ticket" : "the base of an update must be a new realisation");
      return FAMS_EINVAL;
    }
    r->mem = b->x.size() * 64 + (size_t)b->grid.nx * b->grid.ny * 64;   // update work buffers
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->pending.push_back(r);
    *ticket = r->id;
  }
  s->cv_work.notify_all();
  return FAMS_OK;
}

int fams_server_wait(fams_server* s, long long ticket, double timeout_ms, int* done) {
  if (!s || !done) { set_error("null argument"); return FAMS_EINVAL; }
  std::unique_lock<std::mutex> lk(s->mu);
  Request* r = find(s, ticket);
  if (!r) { set_error("unknown ticket"); return FAMS_EINVAL; }
  if (timeout_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                        [&] { return r->done; });
  *done = r->done ? 1 : 0;
  return FAMS_OK;
}

int fams_server_result(fams_server* s, long long ticket, double* x, long long x_cap,
                       double* face_flux, long long face_cap, double* nnc_flux, long long nnc_cap,
                       fams_stats* st, double* latency_ms) {
  if (!s) { set_error("null argument"); return FAMS_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  Request* r = find(s, ticket);
  if (!r) { set_error("unknown ticket"); return FAMS_EINVAL; }
  if (!r->done) { set_error("request not finished"); return FAMS_EINVAL; }
  if (x) {
    if (x_cap < (long long)r->x.size()) { set_error("x buffer too small"); return FAMS_EINVAL; }
    if (int c = copy_out(x, r->x)) return c;
  }
  if (face_flux && !r->face.empty()) {
    if (face_cap < (long long)r->face.size()) { set_error("face buffer too small"); return FAMS_EINVAL; }
    if (int c = copy_out(face_flux, r->face)) return c;
  }
  if (nnc_flux && !r->nnc.empty()) {
    if (nnc_cap < (long long)r->nnc.size()) { set_error("nnc buffer too small"); return FAMS_EINVAL; }
    if (int c = copy_out(nnc_flux, r->nnc)) return c;
  }
  if (st) {
    *st = r->st;
    st->solve_ms = r->t_done - r->t_start;   // service time of its micro-batch
  }
  if (latency_ms) *latency_ms = r->t_done - r->t_submit;
  if (r->status != FAMS_OK) set_error("request failed: " + r->err);
  return r->status;
}

int fams_server_sizes(fams_server* s, long long ticket, long long* n, long long* n_faces,
                      long long* n_nnc) {
  if (!s) { set_error("null argument"); return FAMS_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  Request* r = find(s, ticket);
  if (!r) { set_error("unknown ticket"); return FAMS_EINVAL; }
  if (!r->done) { set_error("request not finished"); return FAMS_EINVAL; }
  if (n) *n = (long long)r->x.size();
  if (n_faces) *n_faces = (long long)r->face.size();
  if (n_nnc) *n_nnc = (long long)r->nnc.size();
  return FAMS_OK;
}

int fams_server_release(fams_server* s, long long ticket) {
  if (!s) { set_error("null argument"); return FAMS_EINVAL; }
  std::vector<fams_ctx*> dead;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Request* r = find(s, ticket);
    if (!r) { set_error("unknown ticket"); return FAMS_EINVAL; }
    if (!r->done) { set_error("request not finished"); return FAMS_EINVAL; }
    // the last released member of an idle resident context frees it
    for (Resident* R : s->residents)
      if (std::find(R->members.begin(), R->members.end(), ticket) != R->members.end()) {
        if (--R->alive == 0 && !R->busy) dead.push_back(retire(s, R));
        break;
      }
    s->all.erase(ticket);
    delete r;
  }
  destroy_all(dead);
  s->cv_work.notify_all();
  return FAMS_OK;
}

void fams_server_destroy(fams_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->all) delete kv.second;   // the workers drained the queue
  for (Resident* R : s->residents) {
    fams_destroy(R->ctx);
    delete R;
  }
  delete s;
}

}  // extern "C"
