// Request server: continuous batching of independent pressure solves.
//
// Callers submit problems (copied at submission) and collect results by
// ticket.  Worker threads, each with its own context and CUDA stream, take
// whatever has arrived -- up to max_batch requests of the oldest request's
// kind (a wide coarse band to factor, or not), and no more than the
// device-memory budget allows next to the micro-batches already in flight --
// set the micro-batch up, solve it and reconstruct its fluxes, while the
// other workers do the same with the requests that arrived in the meantime.
// A request's result does not depend on what it was batched with (one CTA
// per instance in the solve, fixed reduction orders), up to the rounding of
// the coarse operator's atomic sums.  The paper has no counterpart: this is
// the deployment layer around its solver.
#include <chrono>
#include <condition_variable>
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

struct Request {
  long long id = 0;
  fams_grid grid{};
  std::vector<double> perm, xy, kf, rhs;
  fams_fracs fr{};
  fams_opts opts{};
  size_t mem = 0;
  bool heavy = false;   // large coarse factorisation: batched only with its own kind
  // results
  std::vector<double> x, face, nnc;
  fams_stats st{};
  int status = FAMS_OK;
  std::string err;   // detail of a failure
  bool done = false;
  double t_submit = 0, t_start = 0, t_done = 0;
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
// (3D) or three lines (2D) of coarse nodes: a few requests with wide coarse
// bands would otherwise hold a whole micro-batch of small ones
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
  bool stop = false;
  std::vector<std::thread> workers;
};

namespace {

// set up, solve and reconstruct one micro-batch; on a setup failure each
// request is retried alone so that one bad problem fails only itself
void run_batch(fams_server* s, std::vector<Request*>& batch) {
  const int n = (int)batch.size();
  std::vector<fams_grid> grids(n);
  std::vector<const double*> perms(n);
  std::vector<fams_fracs> fracs(n);
  std::vector<fams_opts> opts(n);
  for (int i = 0; i < n; ++i) {
    grids[i] = batch[i]->grid;
    perms[i] = batch[i]->perm.data();
    fracs[i] = batch[i]->fr;
    fracs[i].xy = batch[i]->xy.empty() ? nullptr : batch[i]->xy.data();
    fracs[i].kf = batch[i]->kf.empty() ? nullptr : batch[i]->kf.data();
    opts[i] = batch[i]->opts;
    opts[i].prepare_flux = s->o.with_flux ? 1 : 0;
    batch[i]->t_start = now_ms();
  }
  fams_ctx* ctx = nullptr;
  int st = fams_setup_batch(n, grids.data(), perms.data(), fracs.data(), opts.data(), &ctx);
  if (st != FAMS_OK) {
    if (n > 1) {
      for (Request* r : batch) {
        std::vector<Request*> one{r};
        run_batch(s, one);
      }
    } else {
      batch[0]->status = st;
      batch[0]->err = fams_last_error();
    }
    return;
  }
  std::vector<const double*> rhs(n);
  std::vector<double*> xs(n), faces(n), nncs(n);
  for (int i = 0; i < n; ++i) {
    Request* r = batch[i];
    int nm = 0, nf = 0, nfaces = 0, nnnc = 0;
    fams_sizes(ctx, i, &nm, &nf, nullptr, &nfaces, &nnnc);
    r->x.assign((size_t)nm + nf, 0.0);
    if (!r->rhs.empty() && r->rhs.size() != r->x.size()) r->rhs.resize(r->x.size(), 0.0);
    rhs[i] = r->rhs.empty() ? nullptr : r->rhs.data();
    xs[i] = r->x.data();
    if (s->o.with_flux) {
      r->face.assign((size_t)nfaces, 0.0);
      r->nnc.assign((size_t)std::max(nnnc, 1), 0.0);
      faces[i] = r->face.data();
      nncs[i] = r->nnc.data();
    }
  }
  std::vector<fams_stats> stats(n);
  int ss = fams_solve_batch(ctx, rhs.data(), xs.data(), s->o.tol, stats.data());
  std::string serr = ss == FAMS_OK ? "" : fams_last_error();
  std::vector<int> fst(n, FAMS_OK);
  if (s->o.with_flux && ss != FAMS_ECUDA && ss != FAMS_EINVAL)
    fams_flux_batch(ctx, xs.data(), faces.data(), nncs.data(), fst.data());
  for (int i = 0; i < n; ++i) {
    Request* r = batch[i];
    r->st = stats[i];
    if (ss == FAMS_ECUDA || ss == FAMS_EINVAL || ss == FAMS_ETIMEOUT) r->status = ss;
    else if (!stats[i].converged) r->status = std::isfinite(stats[i].rel_residual) ? FAMS_ENOCONV
                                                                                   : FAMS_EBREAKDOWN;
    else r->status = fst[i];
    if (r->status != FAMS_OK) r->err = r->status == fst[i] ? "flux reconstruction failed" : serr;
  }
  fams_destroy(ctx);
}

void worker(fams_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request*> batch;
    size_t mem = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        if (s->stop) return true;
        if (s->pending.empty()) return false;
        // admission: the first request always fits an idle device
        return s->inflight == 0 || s->inflight + s->pending.front()->mem <= (size_t)s->o.hbm_budget;
      });
      if (s->stop && s->pending.empty()) return;
      // the oldest request, then later ones of the same kind (light or
      // heavy) in arrival order, while they fit
      const bool kind = s->pending.front()->heavy;
      for (auto it = s->pending.begin(); it != s->pending.end() && (int)batch.size() < s->o.max_batch;) {
        Request* r = *it;
        if (r->heavy != kind) { ++it; continue; }
        if (!(s->inflight == 0 && batch.empty()) &&
            s->inflight + mem + r->mem > (size_t)s->o.hbm_budget)
          break;
        batch.push_back(r);
        mem += r->mem;
        it = s->pending.erase(it);
      }
      s->inflight += mem;
    }
    if (batch.empty()) continue;
    run_batch(s, batch);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->inflight -= mem;
      double t = now_ms();
      for (Request* r : batch) {
        r->t_done = t;
        r->done = true;
      }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

Request* find(fams_server* s, long long ticket) {
  auto it = s->all.find(ticket);
  return it == s->all.end() ? nullptr : it->second;
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
  r->perm.assign(perm, perm + cells);
  int nf = fracs ? fracs->n : 0;
  if (nf > 0) {
    if (!fracs->xy || !fracs->kf) {
      delete r;
      set_error("fracture arrays missing");
      return FAMS_EINVAL;
    }
    int w = grid->dim == 3 ? 6 : 4;
    r->xy.assign(fracs->xy, fracs->xy + (size_t)nf * w);
    r->kf.assign(fracs->kf, fracs->kf + nf);
  }
  if (fracs) r->fr = *fracs;
  r->fr.n = nf;
  r->fr.xy = nullptr;
  r->fr.kf = nullptr;
  if (nf == 0) { r->fr.aperture = 1.0; r->fr.h_f = 1.0; }
  r->opts = *opts;
  if (rhs) r->rhs.assign(rhs, rhs + cells);   // matrix sources; fracture sources default to 0
  r->mem = estimate_bytes(*r);
  r->heavy = estimate_heavy(*r);
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
    std::copy(r->x.begin(), r->x.end(), x);
  }
  if (face_flux && !r->face.empty()) {
    if (face_cap < (long long)r->face.size()) { set_error("face buffer too small"); return FAMS_EINVAL; }
    std::copy(r->face.begin(), r->face.end(), face_flux);
  }
  if (nnc_flux && !r->nnc.empty()) {
    if (nnc_cap < (long long)r->nnc.size()) { set_error("nnc buffer too small"); return FAMS_EINVAL; }
    std::copy(r->nnc.begin(), r->nnc.end(), nnc_flux);
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
  std::lock_guard<std::mutex> lk(s->mu);
  Request* r = find(s, ticket);
  if (!r) { set_error("unknown ticket"); return FAMS_EINVAL; }
  if (!r->done) { set_error("request not finished"); return FAMS_EINVAL; }
  s->all.erase(ticket);
  delete r;
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
  delete s;
}

}  // extern "C"
