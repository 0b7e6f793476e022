// Host runtime on top of the C-ABI: the launch-shape autotuner
// (pic_autotune) and the serving loop (pic_server_*).  Only public entry
// points of include/pic.h are used here: this file holds scheduling policy,
// no device code.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/pic.h"
#include "alloc.h"

namespace {

// ------------------------------------------------------------ autotuner --

using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int, int, int, int, long long>;

TuneKey tune_key(const pic_config *c, size_t n) {
  const double cells = (double)c->n[0] * c->n[1];
  const long long ppc = std::llround((double)n / std::max(cells, 1.0));
  const int wstep = c->moving_window ? (c->window_cells > 0 ? c->window_cells : c->patch[0]) : 0;
  return TuneKey(c->dims, c->n[0], c->n[1], c->prec, c->bc_field[0], c->bc_field[1],
                 c->laser_on, c->moving_window, c->filter_passes, wstep, 0, c->tma, ppc);
}

struct TuneEntry {
  int patch[3];
  int block, chunk;
  double ms, ms_given;
  int window_cells;
};

// Key of a plasma-filled workload: the whole grid, boundaries, sources and
// the injection profile (ppc slot -1 marks the plasma form).
TuneKey plasma_key(const pic_config *c) {
  const int wstep = c->moving_window ? (c->window_cells > 0 ? c->window_cells : c->patch[0]) : 0;
  const long long prof = std::llround(c->inj_n0 * 1e9) * 1000003ll + std::llround(c->inj_ramp * 1e3) +
                         7919ll * (c->inj_ppc[0] + 31 * c->inj_ppc[1] + 961 * c->inj_ppc[2]);
  return TuneKey(c->dims, c->n[0], c->n[1], c->prec, c->bc_field[0], c->bc_field[1],
                 c->laser_on, c->moving_window, c->filter_passes, wstep, c->dims == 3 ? c->n[2] : 1,
                 c->tma, -1 - (prof & 0x7fffffffffffll));
}

std::mutex g_tune_mutex;
std::map<TuneKey, TuneEntry> g_tune_cache;

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Time one candidate: a fresh context, the caller's particles, 2 warm-up
// steps, then `steps` timed steps.  Negative on any failure (an invalid
// shape for this grid, an overflow without auto-grow, ...).
double time_candidate(const pic_config &cfg, const double *const p[6], size_t n, int where,
                      int steps) {
  pic_ctx *ctx = nullptr;
  if (pic_create(&cfg, &ctx) != PIC_OK) return -1.0;
  double ms = -1.0;
  if (pic_load_particles(ctx, p[0], p[1], p[2], p[3], p[4], p[5], n, where) == PIC_OK &&
      pic_step(ctx, 2) == PIC_OK) {
    const double t0 = now_ms();
    if (pic_step(ctx, steps) == PIC_OK) ms = (now_ms() - t0) / steps;
  }
  pic_destroy(ctx);
  return ms;
}

// As time_candidate, with the configured plasma filled on the device.
double time_candidate_plasma(const pic_config &cfg, int steps) {
  pic_ctx *ctx = nullptr;
  if (pic_create(&cfg, &ctx) != PIC_OK) return -1.0;
  double ms = -1.0;
  if (pic_load_plasma(ctx) == PIC_OK && pic_step(ctx, 2) == PIC_OK) {
    const double t0 = now_ms();
    if (pic_step(ctx, steps) == PIC_OK) ms = (now_ms() - t0) / steps;
  }
  pic_destroy(ctx);
  return ms;
}

}  // namespace

extern "C" {

void pic_autotune_clear_cache(void) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache.clear();
}

pic_status pic_autotune(const pic_config *cfg, const double *x, const double *y,
                        const double *ux, const double *uy, const double *uz,
                        const double *w, size_t n, int where, int steps, pic_config *tuned,
                        pic_tune_t *out) {
  if (!cfg || !tuned || !out || steps <= 0 || (where != PIC_HOST && where != PIC_DEVICE))
    return PIC_EINVAL;
  if (cfg->dims != 2) return PIC_EINVAL;  // tunes the 2D path
  if (n && (!x || !y || !ux || !uy || !uz || !w)) return PIC_EINVAL;
  if (pic_footprint(cfg, n) == 0) return PIC_EINVAL;  // configuration rejected
  const TuneKey key = tune_key(cfg, n);
  auto apply = [&](const TuneEntry &e, int timed) {
    *tuned = *cfg;
    tuned->patch[0] = e.patch[0];
    tuned->patch[1] = e.patch[1];
    tuned->block = e.block;
    tuned->task_chunk = e.chunk;
    tuned->window_cells = e.window_cells;
    out->patch[0] = e.patch[0];
    out->patch[1] = e.patch[1];
    out->patch[2] = e.patch[2];
    out->block = e.block;
    out->task_chunk = e.chunk;
    out->ms_per_step = e.ms;
    out->ms_given = e.ms_given;
    out->candidates = timed;
  };
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      apply(it->second, 0);
      return PIC_OK;
    }
  }
  const double *p[6] = {x, y, ux, uy, uz, w};
  pic_config base = *cfg;
  base.timing = 0;
  base.use_graph = 1;
  base.auto_grow = 0;  // a replay would be timed too
  base.sort_every = 0;
  base.merge = 0;
  // the configuration as given first: the tuner never returns a slower one
  const double ms_given = time_candidate(base, p, n, where, steps);
  TuneEntry best{{cfg->patch[0], cfg->patch[1], cfg->patch[2]},
                 base.block > 0 ? base.block : 256,
                 base.task_chunk,  // 0: the library's default
                 ms_given, ms_given, cfg->window_cells};
  int timed = 1;
  // the moving window's step (cells) is part of the run: patch widths that
  // divide it keep it, the window then advancing several columns at once
  const int wstep = cfg->window_cells > 0 ? cfg->window_cells : cfg->patch[0];
  for (int P : {8, 16, 32})
    for (int block : {128, 256})
      for (int chunk : {1024, 2048, 4096}) {
        pic_config c = base;
        c.patch[0] = c.patch[1] = P;
        if (c.n[0] % c.patch[0] || c.n[1] % c.patch[1]) continue;
        if (cfg->moving_window) {
          if (wstep % P) continue;
          c.window_cells = wstep;
        }
        c.block = block;
        c.task_chunk = chunk;
        const double ms = time_candidate(c, p, n, where, steps);
        ++timed;
        if (ms > 0 && (best.ms <= 0 || ms < best.ms)) {
          best.patch[0] = c.patch[0];
          best.patch[1] = c.patch[1];
          best.block = block;
          best.chunk = chunk;
          best.window_cells = c.window_cells;
          best.ms = ms;
        }
      }
  if (!(best.ms > 0)) return PIC_ECUDA;  // no candidate ran
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best;
  }
  apply(best, timed);
  return PIC_OK;
}

pic_status pic_autotune_plasma(const pic_config *cfg, int steps, pic_config *tuned,
                               pic_tune_t *out) {
  if (!cfg || !tuned || !out || steps <= 0) return PIC_EINVAL;
  const int dims = cfg->dims;
  if (dims != 2 && dims != 3) return PIC_EINVAL;
  for (int a = 0; a < dims; ++a)
    if (cfg->inj_ppc[a] < 1) return PIC_EINVAL;
  size_t np = 1;
  for (int a = 0; a < dims; ++a) np *= (size_t)cfg->n[a] * cfg->inj_ppc[a];
  if (pic_footprint(cfg, np) == 0) return PIC_EINVAL;  // configuration rejected
  const TuneKey key = plasma_key(cfg);
  auto apply = [&](const TuneEntry &e, int timed) {
    *tuned = *cfg;
    for (int a = 0; a < 3; ++a) tuned->patch[a] = e.patch[a];
    tuned->block = e.block;
    tuned->task_chunk = e.chunk;
    tuned->window_cells = e.window_cells;
    for (int a = 0; a < 3; ++a) out->patch[a] = e.patch[a];
    out->block = e.block;
    out->task_chunk = e.chunk;
    out->ms_per_step = e.ms;
    out->ms_given = e.ms_given;
    out->candidates = timed;
  };
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      apply(it->second, 0);
      return PIC_OK;
    }
  }
  pic_config base = *cfg;
  base.timing = 0;
  base.use_graph = 1;
  base.auto_grow = 0;
  base.sort_every = 0;
  base.merge = 0;
  const double ms_given = time_candidate_plasma(base, steps);
  TuneEntry best{{cfg->patch[0], cfg->patch[1], cfg->patch[2]},
                 base.block > 0 ? base.block : 256,
                 base.task_chunk,  // 0: the library's default
                 ms_given, ms_given, cfg->window_cells};
  int timed = 1;
  const int wstep = cfg->window_cells > 0 ? cfg->window_cells : cfg->patch[0];
  auto consider = [&](pic_config c) {
    for (int a = 0; a < dims; ++a)
      if (c.n[a] % c.patch[a]) return;
    if (cfg->moving_window) {
      if (wstep % c.patch[0]) return;
      c.window_cells = wstep;
    }
    const double ms = time_candidate_plasma(c, steps);
    ++timed;
    if (ms > 0 && (best.ms <= 0 || ms < best.ms)) {
      for (int a = 0; a < 3; ++a) best.patch[a] = c.patch[a];
      best.block = c.block > 0 ? c.block : 256;
      best.chunk = c.task_chunk;
      best.window_cells = c.window_cells;
      best.ms = ms;
    }
  };
  for (int chunk : {1024, 2048, 4096}) {
    if (dims == 2) {
      for (int P : {8, 16, 32})
        for (int block : {128, 256}) {
          pic_config c = base;
          c.patch[0] = c.patch[1] = P;
          c.block = block;
          c.task_chunk = chunk;
          consider(c);
        }
    } else {
      for (int px : {8, 16})
        for (int py : {8, 16})
          for (int pz : {8, 16}) {
            pic_config c = base;
            c.patch[0] = px;
            c.patch[1] = py;
            c.patch[2] = pz;
            c.task_chunk = chunk;
            consider(c);
          }
    }
  }
  if (!(best.ms > 0)) return PIC_ECUDA;  // no candidate ran
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best;
  }
  apply(best, timed);
  return PIC_OK;
}

}  // extern "C"

// --------------------------------------------------------------- server --
//
// Continuous batching over resident runs: FIFO admission by free run slots
// and a device-memory budget (pic_footprint estimates), batched steps of
// every admitted run per tick, retirement at the end of a tick.  The batch
// never references a destroyed context: membership is updated before any
// context is released.

namespace {

struct Request {
  pic_config cfg;
  long long nsteps = 0;
  int keep = 0;
  int state = PIC_REQ_QUEUED;
  int status = PIC_OK;
  long long steps_done = 0, np0 = 0, np = 0;
  size_t footprint = 0;
  double t_submit = 0, t_admit = -1, t_done = -1;
  double U_E = 0, U_B = 0, U_K = 0;
  pic_ctx *ctx = nullptr;
};

}  // namespace

struct pic_server {
  pic_server_config cfg{};
  double t0 = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::map<long long, Request> reqs;
  std::deque<long long> queue;
  std::vector<long long> running;
  // one batch per kind of run: [FP64, FP32] x [default, deterministic]
  pic_batch *batch[4] = {nullptr, nullptr, nullptr, nullptr};
  long long next_id = 1;
  size_t in_use = 0;
  long long ticks = 0, batched_steps = 0, done = 0, failed = 0, submitted = 0, cancelled = 0;
  double particle_steps = 0, busy_s = 0;
};

namespace {

double server_now(const pic_server *s) { return now_ms() * 1e-3 - s->t0; }

// The batch a run belongs to (runs of one batch share precision and the
// deterministic setting).
// The batch a request's run joins: one per precision and mode for 2D runs;
// 3D runs (kSolo3) join none and are stepped one by one in each tick.
constexpr int kSolo3 = 4;
int batch_of(const pic_config &c) {
  if (c.dims == 3) return kSolo3;
  return (c.prec == PIC_FP32 ? 1 : 0) + (c.deterministic ? 2 : 0);
}

// Point each batch at the current running runs of its kind.
pic_status sync_batches(pic_server *s) {
  for (int kind = 0; kind < 4; ++kind) {
    std::vector<pic_ctx *> runs;
    for (long long id : s->running) {
      const Request &r = s->reqs[id];
      if (batch_of(r.cfg) == kind) runs.push_back(r.ctx);
    }
    const pic_status st = pic_batch_set(s->batch[kind], runs.data(), (int)runs.size());
    if (st) return st;
  }
  return PIC_OK;
}

void release(pic_server *s, Request &r) {
  if (r.ctx) pic_destroy(r.ctx);
  r.ctx = nullptr;
  s->in_use -= std::min(s->in_use, r.footprint);
}

void finish(pic_server *s, Request &r, int state, int status) {
  r.state = state;
  r.status = status;
  r.t_done = server_now(s);
  if (state == PIC_REQ_DONE) ++s->done;
  else if (state == PIC_REQ_CANCELLED) ++s->cancelled;
  else ++s->failed;
}

}  // namespace

extern "C" {

pic_status pic_server_create(const pic_server_config *cfg, pic_server **out) {
  if (!cfg || !out) return PIC_EINVAL;
  *out = nullptr;
  if (cfg->max_runs < 0 || cfg->max_runs > PIC_BATCH_MAX || cfg->steps_per_tick < 0)
    return PIC_EINVAL;
  pic_server *s = new (std::nothrow) pic_server();
  if (!s) return PIC_ENOMEM;
  s->cfg = *cfg;
  if (!s->cfg.max_runs) s->cfg.max_runs = PIC_BATCH_MAX;
  if (!s->cfg.steps_per_tick) s->cfg.steps_per_tick = 10;
  s->t0 = now_ms() * 1e-3;
  auto bail = [&](pic_status st) {
    pic_server_destroy(s);
    return st;
  };
  if (cudaSetDevice(cfg->device) != cudaSuccess) return bail(PIC_ECUDA);
  if (cfg->stream) {
    s->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(PIC_ECUDA);
    s->own_stream = true;
  }
  if (!s->cfg.hbm_budget) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return bail(PIC_ECUDA);
    s->cfg.hbm_budget = (size_t)(0.9 * (double)fr);
  }
  for (int kind = 0; kind < 4; ++kind) {
    pic_batch_config bc{};
    bc.stream = s->stream;
    bc.device = cfg->device;
    bc.use_graph = cfg->use_graph;
    const pic_status st = pic_batch_create(&bc, &s->batch[kind]);
    if (st) return bail(st);
  }
  *out = s;
  return PIC_OK;
}

pic_status pic_server_submit(pic_server *s, const pic_config *cfg, long long nsteps, int keep,
                             long long *id) {
  if (!s || !cfg || !id || nsteps <= 0) return PIC_EINVAL;
  if (cfg->dims != 2 && cfg->dims != 3) return PIC_EINVAL;
  for (int a = 0; a < cfg->dims; ++a)
    if (cfg->inj_ppc[a] < 1) return PIC_EINVAL;
  Request r;
  r.cfg = *cfg;
  r.cfg.stream = s->stream;  // one stream for every run and every batch
  r.cfg.device = s->cfg.device;
  size_t np = (size_t)cfg->n[0] * cfg->n[1] * cfg->inj_ppc[0] * cfg->inj_ppc[1];
  if (cfg->dims == 3) np *= (size_t)cfg->n[2] * cfg->inj_ppc[2];
  r.footprint = pic_footprint(&r.cfg, np);
  if (!r.footprint) return PIC_EINVAL;
  r.np0 = (long long)np;
  r.nsteps = nsteps;
  r.keep = keep;
  r.t_submit = server_now(s);
  *id = s->next_id++;
  s->reqs[*id] = r;
  s->queue.push_back(*id);
  ++s->submitted;
  return PIC_OK;
}

pic_status pic_server_tick(pic_server *s, int *running) {
  pic::NvtxRange range("pic_server_tick");
  if (!s) return PIC_EINVAL;
  const double t_enter = server_now(s);
  if (cudaSetDevice(s->cfg.device) != cudaSuccess) return PIC_ECUDA;
  // 1. admission, in arrival order
  bool changed = false;
  while (!s->queue.empty() && (int)s->running.size() < s->cfg.max_runs) {
    Request &r = s->reqs[s->queue.front()];
    if (s->in_use + r.footprint > s->cfg.hbm_budget) {
      if (s->in_use == 0) {  // can never fit
        s->queue.pop_front();
        finish(s, r, PIC_REQ_FAILED, PIC_ENOMEM);
        continue;
      }
      break;
    }
    const long long id = s->queue.front();
    s->queue.pop_front();
    pic_status st = pic_create(&r.cfg, &r.ctx);
    if (st == PIC_OK) st = pic_load_plasma(r.ctx);
    if (st == PIC_OK && r.cfg.dims == 3) {
      // the 3D fill may leave part of the box empty (upper-half plasma)
      pic_diag_t d{};
      st = pic_diag(r.ctx, &d);
      r.np0 = d.np;
    }
    if (st != PIC_OK) {
      if (r.ctx) pic_destroy(r.ctx);
      r.ctx = nullptr;
      finish(s, r, PIC_REQ_FAILED, st);
      continue;
    }
    r.state = PIC_REQ_RUNNING;
    r.t_admit = server_now(s);
    s->in_use += r.footprint;
    s->running.push_back(id);
    changed = true;
  }
  if (changed) {
    const pic_status st = sync_batches(s);
    if (st) return st;
  }
  // 2. batched steps of every admitted run
  if (!s->running.empty()) {
    long long k = s->cfg.steps_per_tick;
    for (long long id : s->running) k = std::min(k, s->reqs[id].nsteps - s->reqs[id].steps_done);
    std::vector<long long> bad;
    for (int kind = 0; kind < 4; ++kind) {
      if (pic_batch_size(s->batch[kind]) == 0) continue;
      const pic_status st = pic_batch_step(s->batch[kind], (int)k);
      if (st == PIC_OK) continue;
      for (long long id : s->running) {
        Request &r = s->reqs[id];
        if (batch_of(r.cfg) == kind && pic_sync(r.ctx) != PIC_OK) {
          r.status = st;
          bad.push_back(id);
        }
      }
    }
    // 3D runs: k steps each on the same stream (no batched 3D kernels)
    for (long long id : s->running) {
      Request &r = s->reqs[id];
      if (batch_of(r.cfg) != kSolo3) continue;
      const pic_status st = pic_step(r.ctx, (int)k);
      if (st != PIC_OK) {
        r.status = st;
        bad.push_back(id);
      }
    }
    s->batched_steps += k;
    for (long long id : s->running) {
      Request &r = s->reqs[id];
      if (std::find(bad.begin(), bad.end(), id) != bad.end()) continue;
      r.steps_done += k;
      s->particle_steps += (double)r.np0 * (double)k;
    }
    // 3. retirement (membership updated before any context is released)
    std::vector<long long> keep_running, leaving;
    for (long long id : s->running) {
      Request &r = s->reqs[id];
      const bool failed = std::find(bad.begin(), bad.end(), id) != bad.end();
      if (failed || r.steps_done >= r.nsteps) leaving.push_back(id);
      else keep_running.push_back(id);
    }
    if (!leaving.empty()) {
      s->running = keep_running;
      const pic_status st = sync_batches(s);
      for (long long id : leaving) {
        Request &r = s->reqs[id];
        if (std::find(bad.begin(), bad.end(), id) != bad.end()) {
          finish(s, r, PIC_REQ_FAILED, r.status ? r.status : PIC_ESTATE);
          release(s, r);
          continue;
        }
        pic_diag_t d{};
        if (pic_diag(r.ctx, &d) == PIC_OK) {
          r.np = d.np;
          r.U_E = d.U_E;
          r.U_B = d.U_B;
          r.U_K = d.U_K;
        }
        finish(s, r, PIC_REQ_DONE, PIC_OK);
        if (!r.keep) release(s, r);
      }
      if (st) return st;
    }
  }
  ++s->ticks;
  s->busy_s += server_now(s) - t_enter;
  if (running) *running = (int)s->running.size();
  return PIC_OK;
}

pic_status pic_server_info(const pic_server *s, long long id, pic_request_info *out) {
  if (!s || !out) return PIC_EINVAL;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return PIC_EINVAL;
  const Request &r = it->second;
  out->state = r.state;
  out->status = r.status;
  out->steps_done = r.steps_done;
  out->steps_total = r.nsteps;
  out->np0 = r.np0;
  out->np = r.np;
  out->footprint = r.footprint;
  out->t_submit = r.t_submit;
  out->t_admit = r.t_admit;
  out->t_done = r.t_done;
  out->U_E = r.U_E;
  out->U_B = r.U_B;
  out->U_K = r.U_K;
  return PIC_OK;
}

pic_status pic_server_take(pic_server *s, long long id, pic_ctx **out) {
  if (!s || !out) return PIC_EINVAL;
  *out = nullptr;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return PIC_EINVAL;
  Request &r = it->second;
  if (r.state != PIC_REQ_DONE || !r.ctx) return PIC_ESTATE;
  *out = r.ctx;
  r.ctx = nullptr;
  s->in_use -= std::min(s->in_use, r.footprint);
  return PIC_OK;
}

pic_status pic_server_cancel(pic_server *s, long long id) {
  if (!s) return PIC_EINVAL;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return PIC_EINVAL;
  Request &r = it->second;
  if (r.state == PIC_REQ_QUEUED) {
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), id));
    finish(s, r, PIC_REQ_CANCELLED, PIC_OK);
    return PIC_OK;
  }
  if (r.state != PIC_REQ_RUNNING) return PIC_ESTATE;
  if (cudaSetDevice(s->cfg.device) != cudaSuccess) return PIC_ECUDA;
  // membership first, then the context goes
  s->running.erase(std::find(s->running.begin(), s->running.end(), id));
  const pic_status st = sync_batches(s);
  finish(s, r, PIC_REQ_CANCELLED, PIC_OK);
  release(s, r);
  return st;
}

pic_status pic_server_get_stats(const pic_server *s, pic_server_stats *out) {
  if (!s || !out) return PIC_EINVAL;
  out->submitted = s->submitted;
  out->done = s->done;
  out->failed = s->failed;
  out->queued = (long long)s->queue.size();
  out->cancelled = s->cancelled;
  out->running = (long long)s->running.size();
  out->ticks = s->ticks;
  out->batched_steps = s->batched_steps;
  out->particle_steps = s->particle_steps;
  out->hbm_in_use = s->in_use;
  out->busy_s = s->busy_s;
  return PIC_OK;
}

double pic_server_clock(const pic_server *s) { return s ? server_now(s) : 0.0; }

void pic_server_destroy(pic_server *s) {
  if (!s) return;
  for (int kind = 0; kind < 4; ++kind)
    if (s->batch[kind]) pic_batch_destroy(s->batch[kind]);
  for (auto &kv : s->reqs)
    if (kv.second.ctx) pic_destroy(kv.second.ctx);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
