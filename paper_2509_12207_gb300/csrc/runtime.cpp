// Serving runtime: chains, frame admission under an HBM budget, and a dispatcher thread that
// releases frames in units (one graph launch each) by the rule in policy.cpp.
//
// Mapping of the paper's mechanisms (Section 4):
//  * urgency evaluation (Eq. 2) at frame arrival and at every release decision; remaining GPU
//    time comes from a lookup table of measured unit durations keyed by (precision, frames in
//    the unit), each entry the mean of its last 8 measurements (Section 4.2, Table 1); the
//    table is seeded by timing every unit size once at creation (the offline profiling stage);
//  * the active kernel buffer (Section 4.4.2) is the list of in-flight units with the chain and
//    urgency they were released with;
//  * task-level stream binding with reservation (Section 4.4.3): every chain owns one stream per
//    priority level; a unit goes to its head frame's chain pool at the level the rule chose;
//  * TH_urgent (Section 4.4.3) is the 95th percentile of the highest urgency seen at each
//    decision during the first frames, unless given;
//  * delayed launching (Section 4.4.4): the dispatcher holds the release and re-checks after the
//    delay quantum or at the next completion;
//  * batched launching with overlap (Section 4.4.5): launches accumulate estimated GPU time into
//    the open batch; when it reaches Delta_eval the batch closes (an event), and releases pause
//    while max_closed closed batches are unfinished;
//  * early chain exit (Section 4.3): frames with negative slack are dropped before release.
// Completion times come from CUDA events (GPU timestamps mapped to the host clock), so latency
// does not depend on how quickly the dispatcher notices a completion.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "pipeline.h"

namespace pp {
namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

constexpr int kLutWindow = 8;
constexpr int kMaxAdmitted = 128;  // admitted-but-unreleased frames per precision, at most

struct Lut {
  double v[kLutWindow] = {0};
  int n = 0, next = 0;
  void add(double x) {
    v[next] = x;
    next = (next + 1) % kLutWindow;
    if (n < kLutWindow) ++n;
  }
  double mean(double dflt) const {
    if (!n) return dflt;
    double s = 0;
    for (int i = 0; i < n; ++i) s += v[i];
    return s / n;
  }
};

constexpr int kMaxSubmit = PP_MAX_SUBMIT;
constexpr int kSynth = 2;       // "precision" class of synthetic-load frames (no pillar model)
constexpr int kSynthUnits = 4;  // units that run synthetic frames

struct Frame {
  uint64_t id = 0;
  int chain = 0, precision = 0;
  double t_arr = 0, deadline = 0, t_release = 0;
  int64_t n = 0;
  const float* src = nullptr;  // device pointer (borrowed) or pinned staging slot
  int staging = -1;
  int rslot = -1;              // result pool slot (reserved at admission)
  int unit = -1, slot = -1;
  bool dropped = false, done = false, polled = false;
  double delay_start = -1;
  double est_scale = 1.0;      // estimate-noise factor (1 unless the experiment is on)
  bool pinned = false;         // borrowed page-locked host memory (read over the host link)
  char* hout_dev = nullptr;    // caller's page-locked result buffer: device view, host pointer
  void* hout_host = nullptr;
};

struct Unit {
  Pipeline pipe;
  int precision = 0;
  bool busy = false, running = false;
  bool failed = false;  // the launch itself failed: its frames complete with PP_FRAME_ERROR
  int nf = 0, level = 0, head_chain = 0;
  uint64_t frames[8] = {0};
  cudaEvent_t start = nullptr, done = nullptr;
  double ul = 0, est = 0, t_launch = 0;
};

struct Chain {
  bool used = false;
  double period_ms = 0, deadline_ms = 0;
  int precision = 0;              // PP_F32 / PP_BF16, or kSynth for a synthetic-load chain
  // synthetic load: n_kernels launches of synth_ctas CTAs x synth_iters passes per frame, and
  // the chain's own duration estimates (its frames are not interchangeable with other chains')
  int n_kernels = 0, synth_ctas = 0, synth_iters = 0;
  double kernel_us = 0, util = 1.0;  // util: fraction of the SMs its kernels occupy
  Lut lut;
  std::vector<cudaStream_t> streams;  // one per priority level, level 0 highest
  uint64_t frames = 0, missed = 0;
  std::vector<double> lat;
};

}  // namespace
}  // namespace pp

using namespace pp;

struct pp_ctx {
  pp_config cfg{};
  int device = 0;
  int num_pri = 1, prio_greatest = 0;
  Model models[2];
  bool have[3] = {false, false, false};  // [kSynth]: synthetic-load units exist
  std::vector<Unit*> units;
  int capacity[3] = {0, 0, 0}, admitted[3] = {0, 0, 0};
  SynthBuf synth;
  int synth_first = -1;  // index of the first synthetic unit in `units`
  Chain chains[PP_MAX_CHAINS];
  std::map<uint64_t, Frame*> frames;
  std::vector<Frame*> ready;
  std::deque<pp_result> completed;
  std::vector<float*> staging;
  std::vector<int> staging_free;
  // per-precision result pools: every admitted frame owns one slot until it is released, so
  // units are free again as soon as they complete
  struct Pool {
    void* base = nullptr;
    size_t slot_bytes = 0;
    std::vector<size_t> block_off;
    std::vector<int> free;
  } pool[3];                     // [kSynth] stays empty: synthetic frames have no outputs
  Lut lut[2][9];
  // batched synchronisation gate
  double open_sum = 0;
  std::vector<int> open_units;
  std::deque<std::vector<int>> closed;
  // urgency threshold
  double th = -1;
  std::vector<double> th_samples;
  bool calibrating = false;
  // timing reference: GPU event <-> host clock
  cudaEvent_t ref_event = nullptr;
  double ref_host = 0;
  cudaStream_t aux = nullptr;
  cudaStream_t notify = nullptr;  // completion callbacks, so that no unit stream waits on the host
  // stats
  uint64_t submitted = 0, n_done = 0, n_dropped = 0, n_missed = 0, rejected = 0, launched = 0;
  uint64_t batch_frames = 0, delayed = 0, collisions = 0, decisions = 0;
  double delayed_us = 0, sched_us = 0, first_arr = -1, last_done = -1;
  std::vector<double> lat_all;
  uint64_t next_id = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread dispatcher;
  std::atomic<bool> stop{false};
  uint64_t device_errors = 0;      // units whose launch or device work failed
  unsigned device_error_code = 0;  // the last nonzero device error word a unit reported
  // decision log (cfg.decision_log > 0): every release decision the dispatcher takes, with the
  // inputs it took it on, until the log holds cfg.decision_log records
  std::vector<pp_decision_record> log;
  std::vector<pp_policy_frame> log_ready;
  std::vector<pp_policy_active> log_active;
  std::vector<uint64_t> log_drops;
};

namespace {

double unit_est(pp_ctx* c, int prec, int nf) {
  return c->lut[prec][nf].mean(c->lut[prec][1].mean(1000.0) * nf);
}

// GPU-time estimate of one frame alone (before any estimate noise)
double frame_est(pp_ctx* c, const Frame* f) {
  if (f->precision == kSynth) {
    const Chain& ch = c->chains[f->chain];
    return ch.lut.mean(ch.n_kernels * ch.kernel_us);
  }
  return unit_est(c, f->precision, 1);
}

void CUDART_CB notify_cb(void* p) {
  pp_ctx* c = static_cast<pp_ctx*>(p);
  c->cv_work.notify_one();
}

double event_host_time(pp_ctx* c, cudaEvent_t e) {
  float ms = 0;
  if (cudaEventElapsedTime(&ms, c->ref_event, e) != cudaSuccess) {
    cudaGetLastError();
    return now_us();
  }
  return c->ref_host + (double)ms * 1000.0;
}

void push_result(pp_ctx* c, Frame* f, int status, double t_done) {
  pp_result r;
  memset(&r, 0, sizeof(r));
  r.frame_id = f->id;
  r.chain_id = f->chain;
  r.status = status;
  r.t_arr_us = f->t_arr;
  r.t_release_us = f->t_release;
  r.t_done_us = t_done;
  r.deadline_us = f->deadline;
  r.missed = status != PP_FRAME_DONE || t_done > f->deadline;
  Chain& ch = c->chains[f->chain];
  ch.frames++;
  if (r.missed) {
    ch.missed++;
    c->n_missed++;
  }
  if (status == PP_FRAME_DONE) {
    const double lat = t_done - f->t_arr;
    ch.lat.push_back(lat);
    c->lat_all.push_back(lat);
    c->n_done++;
    if (t_done > c->last_done) c->last_done = t_done;
    Unit* u = c->units[f->unit];
    r.batch = u->nf;
    r.level = u->level;
    if (f->precision == kSynth) {
      r.out_dtype = -1;  // synthetic load: timing only, no outputs
    } else {
      const Model* m = u->pipe.model();
      const pp_ctx::Pool& pl = c->pool[f->precision];
      char* base = static_cast<char*>(pl.base) + (size_t)f->rslot * pl.slot_bytes;
      r.out_dtype = m->precision;
      if (m->head_outputs > 0) {
        r.out_dev = base + pl.block_off[0];
        r.out_c = m->head_c;
        r.out_valid_c = m->head_outputs;
        r.out_h = m->out_h();
        r.out_w = m->out_w();
      }
      const std::vector<int> kept = m->kept_blocks();
      for (size_t k = 0; k < kept.size(); ++k) {
        const int b = kept[k];
        const LayerSpec& L = m->layers[m->block_end[b]];
        r.block_dev[b] = base + pl.block_off[k];
        r.block_c[b] = L.cout;
        r.block_h[b] = L.Ho;
        r.block_w[b] = L.Wo;
        r.out_dev = r.block_dev[b];
        r.out_c = r.out_valid_c = L.cout;
        r.out_h = L.Ho;
        r.out_w = L.Wo;
      }
      r.num_pillars = u->pipe.num_pillars_host()[f->slot];
      r.out_host = f->hout_host;  // the final output's host copy, if the caller gave a buffer
    }
  } else {
    c->n_dropped += status == PP_FRAME_DROPPED;
  }
  f->done = true;
  c->completed.push_back(r);
  c->cv_done.notify_all();
}

void free_staging(pp_ctx* c, Frame* f) {
  if (f->staging >= 0) {
    c->staging_free.push_back(f->staging);
    f->staging = -1;
  }
}

void free_result(pp_ctx* c, Frame* f) {
  if (f->rslot >= 0) {
    c->pool[f->precision].free.push_back(f->rslot);
    f->rslot = -1;
  }
}

// Completed units: results, estimate table, batch gate.  The unit is free again at once.
void reap(pp_ctx* c) {
  for (size_t ui = 0; ui < c->units.size(); ++ui) {
    Unit* u = c->units[ui];
    if (!u->running) continue;
    const cudaError_t q = cudaEventQuery(u->done);
    if (q == cudaErrorNotReady) continue;
    u->running = false;
    u->busy = false;
    if (q != cudaSuccess) cudaGetLastError();
    // a unit failed if its launch did, if its event reports an error, or if its last kernel
    // saw a device error word set (a conv whose bounded wait ran out skipped its stores, and
    // every conv after it exits at once): its frames' outputs are not to be trusted
    unsigned code = 0;
    if (!u->failed && q == cudaSuccess && u->precision != kSynth) code = u->pipe.device_error_host();
    const bool ok = !u->failed && q == cudaSuccess && code == 0;
    u->failed = false;
    if (!ok) {
      c->device_errors++;
      if (code) c->device_error_code = code;
    }
    const double t_done = q == cudaSuccess ? event_host_time(c, u->done) : now_us();
    float ms = 0;
    // only a unit that ran to completion feeds the estimate table
    if (ok && cudaEventElapsedTime(&ms, u->start, u->done) == cudaSuccess) {
      if (u->precision == kSynth)
        c->chains[u->head_chain].lut.add(ms * 1000.0);
      else
        c->lut[u->precision][u->nf].add(ms * 1000.0);
    } else
      cudaGetLastError();
    for (int i = 0; i < u->nf; ++i) {
      Frame* f = c->frames[u->frames[i]];
      free_staging(c, f);
      push_result(c, f, ok ? PP_FRAME_DONE : PP_FRAME_ERROR, t_done);
    }
    // batch gate: closed batches finish in launch order
    const int id = (int)ui;
    for (auto& b : c->closed) b.erase(std::remove(b.begin(), b.end(), id), b.end());
    while (!c->closed.empty() && c->closed.front().empty()) c->closed.pop_front();
    c->open_units.erase(std::remove(c->open_units.begin(), c->open_units.end(), id), c->open_units.end());
  }
}

int closed_pending(pp_ctx* c) {
  int n = 0;
  for (auto& b : c->closed) n += !b.empty();
  return n;
}

// One stream per priority level for a new chain, level 0 the highest.
int chain_streams(pp_ctx* c, Chain* ch) {
  for (int l = 0; l < c->num_pri; ++l) {
    cudaStream_t s;
    int st = cuda_status(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, c->prio_greatest + l),
                         "chain stream");
    if (st) return st;
    ch->streams.push_back(s);
  }
  return PP_OK;
}

int free_unit(pp_ctx* c, int prec) {
  for (size_t i = 0; i < c->units.size(); ++i)
    if (!c->units[i]->busy && c->units[i]->precision == prec) return (int)i;
  return -1;
}

pp_policy_config policy_cfg(pp_ctx* c) {
  pp_policy_config p;
  p.policy = c->cfg.policy;
  p.max_batch = c->cfg.max_batch;
  p.max_closed = c->cfg.max_closed;
  p.num_pri = c->num_pri;
  p.early_exit = c->cfg.early_exit;
  p.th_urgent = c->th;
  p.util_exempt = c->cfg.util_exempt;
  p.eqdf_lambda = c->cfg.eqdf_lambda;
  return p;
}

// A ready frame as the release rule sees it: one unit's estimate remains; its utilisation (1.0
// for pillar frames, whose kernels fill the GPU, so the delay exemption never applies to them;
// a synthetic chain's SM fraction); its chain's period.
pp_policy_frame policy_frame(pp_ctx* c, const Frame* f) {
  pp_policy_frame p;
  p.frame_id = f->id;
  p.chain_id = f->chain;
  p.precision = f->precision;
  p.t_arr_us = f->t_arr;
  p.deadline_us = f->deadline;
  p.est_gpu_us = frame_est(c, f) * f->est_scale;
  p.est_cpu_us = 0.0;
  p.util = c->chains[f->chain].util;
  p.period_us = c->chains[f->chain].period_ms * 1000.0;
  return p;
}

int launch_unit(pp_ctx* c, const pp_policy_decision& d, double t) {
  Frame* head = c->frames[d.frames[0]];
  const int prec = head->precision;
  const int ui = free_unit(c, prec);
  if (ui < 0) return 1;  // every unit of this precision is busy: wait for a completion/release
  Unit* u = c->units[ui];
  const float* srcs[kMaxUnit];
  int counts[kMaxUnit];
  bool direct[kMaxUnit], host_mapped[kMaxUnit];
  char* dsts[kMaxUnit];
  char* hdsts[kMaxUnit];
  const pp_ctx::Pool& pl = c->pool[prec];
  // a synthetic frame runs alone: its chain's kernels are its own (the rest stay ready)
  const int nf = prec == kSynth ? 1 : d.n_frames;
  u->nf = nf;
  u->level = d.level;
  u->head_chain = head->chain;
  {
    // the unit's priority when released (urgency UL for the urgency policy)
    const pp_policy_config pc = policy_cfg(c);
    const pp_policy_frame hf = policy_frame(c, head);
    u->ul = pp_policy_priority(&pc, t, &hf);
  }
  u->est = prec == kSynth ? frame_est(c, head) : unit_est(c, prec, nf);
  for (int i = 0; i < nf; ++i) {
    Frame* f = c->frames[d.frames[i]];
    u->frames[i] = f->id;
    f->unit = ui;
    f->slot = i;
    f->t_release = t;
    srcs[i] = f->src;
    counts[i] = (int)f->n;
    direct[i] = f->staging < 0;  // a borrowed buffer is read in place
    host_mapped[i] = f->pinned;  // ... over the host link, once
    dsts[i] = f->rslot < 0 ? nullptr : static_cast<char*>(pl.base) + (size_t)f->rslot * pl.slot_bytes;
    hdsts[i] = f->hout_dev;
    if (f->delay_start >= 0) {
      c->delayed_us += t - f->delay_start;
      f->delay_start = -1;
    }
    c->ready.erase(std::remove(c->ready.begin(), c->ready.end(), f), c->ready.end());
  }
  // collision: a launch while another chain's urgent unit is in flight (or this one is urgent)
  if (c->th > 0) {
    for (Unit* o : c->units)
      if (o->running && o->head_chain != u->head_chain && (o->ul > c->th || u->ul > c->th)) {
        c->collisions++;
        break;
      }
  }
  const int lvl = std::min(std::max(d.level, 0), c->num_pri - 1);
  cudaStream_t s = c->chains[head->chain].streams[lvl];
  u->busy = true;
  u->running = true;
  u->t_launch = t;
  int st = cuda_status(cudaEventRecord(u->start, s), "record start");
  if (!st && prec == kSynth) {
    const Chain& ch = c->chains[head->chain];
    st = synth_launch(c->synth, ui - c->synth_first, ch.synth_ctas, ch.synth_iters, ch.n_kernels, s);
  } else if (!st) {
    // the unit's graph also copies every frame's block outputs into its result slot
    st = u->pipe.run(nf, srcs, counts, direct, dsts, c->cfg.use_graphs != 0, s, host_mapped, hdsts);
  }
  // the completion event is recorded even after a failed launch, so that reap() sees this
  // launch's end (not an earlier one's) and the unit is not reused while work it did enqueue
  // may still run; the frames then complete with PP_FRAME_ERROR
  const int rec = cuda_status(cudaEventRecord(u->done, s), "record done");
  if (!st) st = rec;
  u->failed = st != 0;
  if (u->failed) {
    cudaGetLastError();
    if (rec) {
      // not even the event could be recorded: nothing of this launch can be waited for, so
      // finish its frames now (the unit stays out of use: its stream may hold work)
      u->running = false;
      u->failed = false;
      c->device_errors++;
      for (int i = 0; i < nf; ++i) {
        Frame* f = c->frames[u->frames[i]];
        free_staging(c, f);
        push_result(c, f, PP_FRAME_ERROR, t);
      }
      return 0;
    }
  } else {
    // wake the dispatcher at completion from a separate stream: a host function in the unit's
    // own stream would hold back whatever is queued behind it there until the callback has run
    // (without it the dispatcher still looks every 500 us while a unit runs)
    if (cudaStreamWaitEvent(c->notify, u->done, 0) != cudaSuccess ||
        cudaLaunchHostFunc(c->notify, notify_cb, c) != cudaSuccess)
      cudaGetLastError();
  }
  c->launched++;
  c->batch_frames += nf;
  if (u->failed) return 0;  // no estimate accounting for a launch that did not happen
  // batched synchronisation bookkeeping
  c->open_units.push_back(ui);
  c->open_sum += u->est;
  if (c->open_sum >= c->cfg.delta_eval_us) {
    c->closed.push_back(c->open_units);
    c->open_units.clear();
    c->open_sum = 0;
  }
  return 0;
}

void calibrate(pp_ctx* c, double t) {
  if (!c->calibrating) return;
  double mx = -INFINITY;
  for (Frame* f : c->ready) {
    const double s = f->deadline - frame_est(c, f) * f->est_scale - t;
    if (s > 0) mx = std::max(mx, 1.0 / s);
  }
  for (Unit* u : c->units)
    if (u->running) mx = std::max(mx, u->ul);
  if (std::isfinite(mx)) c->th_samples.push_back(mx);
  if ((int64_t)c->n_done >= c->cfg.th_calib_frames && c->th_samples.size() >= 8) {
    std::vector<double> v = c->th_samples;
    std::sort(v.begin(), v.end());
    c->th = v[(size_t)std::floor(0.95 * (double)(v.size() - 1))];
    c->calibrating = false;
  }
}

// One pass of decisions; returns the time (us) until the dispatcher should look again.
double decide_all(pp_ctx* c) {
  double wake = 1e9;
  for (int guard = 0; guard < 1024; ++guard) {
    const double t = now_us();
    calibrate(c, t);
    std::vector<pp_policy_frame> rf;
    rf.reserve(c->ready.size());
    for (Frame* f : c->ready) rf.push_back(policy_frame(c, f));
    std::vector<pp_policy_active> act;
    for (Unit* u : c->units)
      if (u->running) act.push_back({u->head_chain, u->ul});
    pp_policy_config pc = policy_cfg(c);
    pp_policy_decision d;
    std::vector<uint64_t> drops(rf.size() + 1);
    const int pend = closed_pending(c);
    pp_policy_decide(&pc, t, rf.data(), (int)rf.size(), act.data(), (int)act.size(), pend, &d,
                     drops.data(), (int)drops.size());
    pp_decision_record* rec = nullptr;
    if ((int64_t)c->log.size() < (int64_t)c->cfg.decision_log) {
      pp_decision_record r;
      memset(&r, 0, sizeof(r));
      r.t_us = t;
      r.cfg = pc;
      r.closed_pending = pend;
      r.n_ready = (int)rf.size();
      r.n_active = (int)act.size();
      r.ready_off = (int64_t)c->log_ready.size();
      r.active_off = (int64_t)c->log_active.size();
      r.drops_off = (int64_t)c->log_drops.size();
      r.decision = d;
      c->log_ready.insert(c->log_ready.end(), rf.begin(), rf.end());
      c->log_active.insert(c->log_active.end(), act.begin(), act.end());
      c->log_drops.insert(c->log_drops.end(), drops.begin(), drops.begin() + d.n_drops);
      c->log.push_back(r);
      rec = &c->log.back();
    }
    for (int i = 0; i < d.n_drops; ++i) {
      Frame* f = c->frames[drops[i]];
      c->ready.erase(std::remove(c->ready.begin(), c->ready.end(), f), c->ready.end());
      f->dropped = true;
      free_staging(c, f);
      free_result(c, f);
      c->admitted[f->precision]--;
      push_result(c, f, PP_FRAME_DROPPED, t);
    }
    c->decisions++;
    if (d.kind == PP_DECIDE_RELEASE) {
      if (launch_unit(c, d, t)) return 200.0;  // no free unit
      if (rec) rec->launched = 1;
      c->sched_us += now_us() - t;
      continue;
    }
    c->sched_us += now_us() - t;
    if (d.kind == PP_DECIDE_DELAY) {
      for (Frame* f : c->ready)
        if (f->delay_start < 0) {
          f->delay_start = t;
          c->delayed++;
        }
      wake = std::min(wake, c->cfg.delay_quantum_us);
    } else if (d.kind == PP_DECIDE_WAIT) {
      wake = std::min(wake, 200.0);
    }
    break;
  }
  bool running = false;
  for (Unit* u : c->units) running |= u->running;
  if (running) wake = std::min(wake, 500.0);
  return wake;
}

void dispatcher_main(pp_ctx* c) {
  cudaSetDevice(c->device);
  std::unique_lock<std::mutex> lk(c->mu);
  while (!c->stop.load()) {
    reap(c);
    const double wake = decide_all(c);
    c->cv_work.wait_for(lk, std::chrono::microseconds((int64_t)std::max(20.0, std::min(wake, 1e6))));
  }
}

void destroy_units(pp_ctx* c) {
  for (Unit* u : c->units) {
    u->pipe.release();
    if (u->start) cudaEventDestroy(u->start);
    if (u->done) cudaEventDestroy(u->done);
    delete u;
  }
  c->units.clear();
  for (int p = 0; p < 2; ++p)
    if (c->have[p]) c->models[p].release();
  for (float* s : c->staging) cudaFreeHost(s);
  c->staging.clear();
  synth_free(&c->synth);
  for (auto& pl : c->pool)
    if (pl.base) cudaFree(pl.base);
  for (auto& ch : c->chains)
    for (cudaStream_t s : ch.streams) cudaStreamDestroy(s);
  if (c->ref_event) cudaEventDestroy(c->ref_event);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->notify) cudaStreamDestroy(c->notify);
  for (auto& kv : c->frames) delete kv.second;
  c->frames.clear();
}

}  // namespace

extern "C" {

double pp_now_us(void) { return now_us(); }

size_t pp_struct_size(const char* name) {
  if (!name) return 0;
  static const struct {
    const char* n;
    size_t s;
  } kSizes[] = {{"pp_config", sizeof(pp_config)},
                {"pp_result", sizeof(pp_result)},
                {"pp_stats", sizeof(pp_stats)},
                {"pp_geometry", sizeof(pp_geometry)},
                {"pp_arrival", sizeof(pp_arrival)},
                {"pp_replay_stats", sizeof(pp_replay_stats)},
                {"pp_policy_frame", sizeof(pp_policy_frame)},
                {"pp_policy_active", sizeof(pp_policy_active)},
                {"pp_policy_config", sizeof(pp_policy_config)},
                {"pp_policy_decision", sizeof(pp_policy_decision)},
                {"pp_decision_record", sizeof(pp_decision_record)}};
  for (const auto& e : kSizes)
    if (strcmp(e.n, name) == 0) return e.s;
  return 0;
}

double pp_noise_factor(uint64_t seed, uint64_t frame_id, double eps) {
  uint64_t z = seed + frame_id * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  return 1.0 + eps * (2.0 * u - 1.0);
}

void pp_config_defaults(pp_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->max_batch = 8;
  cfg->cap_points = 150000;
  cfg->precisions = 3;
  cfg->units = 0;
  cfg->hbm_budget_bytes = 20ull << 30;
  cfg->policy = PP_POLICY_URGENCY;
  cfg->use_graphs = 1;
  cfg->delta_eval_us = 500.0;
  cfg->max_closed = 2;
  cfg->delay_quantum_us = 1000.0;
  cfg->th_urgent = 0.0;
  cfg->th_calib_frames = 64;
  cfg->util_exempt = 0.1;
  cfg->early_exit = 1;
  cfg->num_streams = 0;
  cfg->autotune = 1;
  cfg->stream_k = 0;
  cfg->head_outputs = 0;
  cfg->up_channels = 128;
  cfg->eqdf_lambda = 0.5;
}

int pp_create(const pp_config* cfg, pp_ctx** out) {
  if (!cfg || !out) return fail(PP_EINVAL, "create: NULL argument");
  if (cfg->max_batch < 1 || cfg->max_batch > 8) return fail(PP_EINVAL, "create: max_batch must be 1..8");
  if (cfg->cap_points < 1 || cfg->cap_points > (1 << 24)) return fail(PP_EINVAL, "create: cap_points 1..2^24");
  if ((cfg->precisions & 3) == 0) return fail(PP_EINVAL, "create: no precision enabled");
  if (cfg->policy < PP_POLICY_FIFO || cfg->policy > PP_POLICY_EQDF) return fail(PP_EINVAL, "create: bad policy");
  if (!std::isfinite(cfg->eqdf_lambda)) return fail(PP_EINVAL, "create: eqdf_lambda must be finite");
  if (!(cfg->est_noise >= 0 && cfg->est_noise < 1)) return fail(PP_EINVAL, "create: est_noise must be in [0, 1)");
  if (cfg->units < 0 || cfg->units > 64 || cfg->max_closed < 0 || !(cfg->delta_eval_us >= 0) ||
      cfg->max_admitted < 0 ||
      !(cfg->delay_quantum_us > 0) || cfg->th_calib_frames < 0 || cfg->decision_log < 0 ||
      cfg->decision_log > (1 << 20))
    return fail(PP_EINVAL, "create: bad runtime knob");
  pp_ctx* c = new (std::nothrow) pp_ctx();
  if (!c) return fail(PP_ENOMEM, "create: host allocation");
  c->cfg = *cfg;
  c->cfg.pfn_w = c->cfg.pfn_bn = nullptr;  // not retained: weights are copied to the device
  c->cfg.conv_w = c->cfg.conv_bn = nullptr;
  int st = cuda_status(cudaGetDevice(&c->device), "get device");
  int least = 0, greatest = 0;
  if (!st) st = cuda_status(cudaDeviceGetStreamPriorityRange(&least, &greatest), "priority range");
  c->prio_greatest = greatest;
  c->num_pri = least - greatest + 1;
  if (cfg->num_streams > 0) c->num_pri = std::min(c->num_pri, cfg->num_streams);
  if (!st) st = cuda_status(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking), "aux stream");
  if (!st) st = cuda_status(cudaStreamCreateWithFlags(&c->notify, cudaStreamNonBlocking), "notify stream");
  uint64_t used = 0;
  for (int p = 0; p < 2 && !st; ++p) {
    if (!(cfg->precisions & (1 << p))) continue;
    st = c->models[p].upload(cfg, p, c->aux);
    c->have[p] = st == PP_OK;
    used += c->models[p].bytes;
  }
  // units: round-robin over precisions while the budget allows
  const int want = cfg->units > 0 ? cfg->units : 16;
  for (int k = 0; k < want && !st; ++k) {
    for (int p = 0; p < 2 && !st; ++p) {
      if (!c->have[p]) continue;
      Unit* u = new (std::nothrow) Unit();
      if (!u) { st = fail(PP_ENOMEM, "create: host allocation"); break; }
      u->precision = p;
      // the first unit of each precision tunes the conv tiles; later units reuse the table
      st = u->pipe.init(&c->models[p], cfg->max_batch, cfg->cap_points, cfg->use_graphs != 0,
                        cfg->autotune != 0 && k == 0, cfg->stream_k != 0, c->aux);
      if (!st) st = cuda_status(cudaEventCreate(&u->start), "event");
      if (!st) st = cuda_status(cudaEventCreate(&u->done), "event");
      if (!st && used + u->pipe.bytes() > cfg->hbm_budget_bytes) {
        u->pipe.release();
        cudaEventDestroy(u->start);
        cudaEventDestroy(u->done);
        delete u;
        if (c->capacity[p] == 0) st = fail(PP_ENOMEM, "create: one unit (precision %d) exceeds the HBM budget", p);
        k = want;  // budget exhausted
        break;
      }
      if (st) { u->pipe.release(); delete u; break; }
      used += u->pipe.bytes();
      c->units.push_back(u);
      c->capacity[p] += cfg->max_batch;
    }
  }
  // result pools: one slot per admissible frame, from what is left of the budget
  for (int p = 0; p < 2 && !st; ++p) {
    if (!c->have[p] || c->capacity[p] == 0) continue;
    pp_ctx::Pool& pl = c->pool[p];
    pl.slot_bytes = c->models[p].result_layout(&pl.block_off);
    c->capacity[p] = 0;
  }
  {
    const uint64_t left = cfg->hbm_budget_bytes > used ? cfg->hbm_budget_bytes - used : 0;
    const uint64_t per = c->pool[0].slot_bytes + c->pool[1].slot_bytes;
    const uint64_t cap = cfg->max_admitted > 0 ? (uint64_t)std::min(cfg->max_admitted, kMaxAdmitted)
                                               : (uint64_t)kMaxAdmitted;
    int n = per ? (int)std::min<uint64_t>(left / per, cap) : 0;
    for (int p = 0; p < 2 && !st; ++p) {
      pp_ctx::Pool& pl = c->pool[p];
      if (!pl.slot_bytes) continue;
      if (n < 1) st = fail(PP_ENOMEM, "create: no room for a result slot in the budget");
      if (!st) st = cuda_status(cudaMalloc(&pl.base, pl.slot_bytes * (size_t)n), "result pool");
      // zero once: the last conv writes a slot's interior directly, so its border must stay zero
      if (!st) st = cuda_status(cudaMemsetAsync(pl.base, 0, pl.slot_bytes * (size_t)n, c->aux), "clear result pool");
      for (int i = 0; i < n && !st; ++i) pl.free.push_back(n - 1 - i);
      c->capacity[p] = n;
      used += pl.slot_bytes * (size_t)n;
    }
  }
  // pinned staging for host submissions: one slot per admissible frame
  const int slots = c->capacity[0] + c->capacity[1];
  for (int i = 0; i < slots && !st; ++i) {
    float* s = nullptr;
    st = cuda_status(cudaMallocHost(&s, (size_t)cfg->cap_points * 16), "pinned staging");
    if (!st) {
      c->staging.push_back(s);
      c->staging_free.push_back(i);
    }
  }
  // offline profiling: time every unit size once to seed the estimate table
  for (int p = 0; p < 2 && !st; ++p) {
    const int ui = free_unit(c, p);
    if (ui < 0) continue;
    Unit* u = c->units[ui];
    const float* srcs[kMaxUnit] = {nullptr};
    int counts[kMaxUnit] = {0};
    char* dsts[kMaxUnit];  // free result slots: the timing includes the result copies
    const pp_ctx::Pool& pl = c->pool[p];
    for (int i = 0; i < kMaxUnit; ++i)
      dsts[i] = static_cast<char*>(pl.base) + (size_t)(i % c->capacity[p]) * pl.slot_bytes;
    for (int b = 1; b <= cfg->max_batch && !st; ++b) {
      for (int rep = 0; rep < 2 && !st; ++rep) {
        st = cuda_status(cudaEventRecord(u->start, c->aux), "profile");
        if (!st) st = u->pipe.run(b, srcs, counts, nullptr, dsts, cfg->use_graphs != 0, c->aux);
        if (!st) st = cuda_status(cudaEventRecord(u->done, c->aux), "profile");
        if (!st) st = cuda_status(cudaEventSynchronize(u->done), "profile");
        float ms = 0;
        if (!st && rep == 1 && cudaEventElapsedTime(&ms, u->start, u->done) == cudaSuccess)
          c->lut[p][b].add(ms * 1000.0);
      }
    }
  }
  if (!st) st = cuda_status(cudaEventCreate(&c->ref_event), "ref event");
  if (!st) st = cuda_status(cudaEventRecord(c->ref_event, c->aux), "ref event");
  if (!st) st = cuda_status(cudaEventSynchronize(c->ref_event), "ref event");
  c->ref_host = now_us();
  if (st) {
    destroy_units(c);
    delete c;
    return st;
  }
  c->th = cfg->th_urgent > 0 ? cfg->th_urgent : -1.0;
  c->calibrating = cfg->th_urgent == 0.0 && cfg->policy == PP_POLICY_URGENCY;
  c->dispatcher = std::thread(dispatcher_main, c);
  *out = c;
  return PP_OK;
}

int pp_register_chain(pp_ctx* c, int32_t chain_id, double period_ms, double rel_deadline_ms,
                      int32_t precision) {
  if (!c || chain_id < 0 || chain_id >= PP_MAX_CHAINS || !(rel_deadline_ms > 0) || !(period_ms > 0))
    return fail(PP_EINVAL, "register_chain: bad argument");
  if (precision != PP_F32 && precision != PP_BF16) return fail(PP_EINVAL, "register_chain: bad precision");
  std::lock_guard<std::mutex> lk(c->mu);
  if (!c->have[precision]) return fail(PP_EINVAL, "register_chain: precision %d not enabled", precision);
  Chain& ch = c->chains[chain_id];
  if (ch.used) return fail(PP_ESTATE, "register_chain: chain %d already registered", chain_id);
  int st = chain_streams(c, &ch);
  if (st) return st;
  ch.used = true;
  ch.period_ms = period_ms;
  ch.deadline_ms = rel_deadline_ms;
  ch.precision = precision;
  return PP_OK;
}

int pp_register_synthetic_chain(pp_ctx* c, int32_t chain_id, double period_ms, double rel_deadline_ms,
                                int32_t n_kernels, double kernel_us, double util) {
  if (!c || chain_id < 0 || chain_id >= PP_MAX_CHAINS || !(rel_deadline_ms > 0) || !(period_ms > 0) ||
      n_kernels < 1 || n_kernels > 256 || !(kernel_us >= 1 && kernel_us <= 100000) || !(util > 0 && util <= 1) ||
      n_kernels * kernel_us > 1e6)
    return fail(PP_EINVAL, "register_synthetic_chain: bad argument (1..256 kernels of 1 us..100 ms, util (0, 1], "
                           "at most 1 s per frame)");
  std::lock_guard<std::mutex> lk(c->mu);
  Chain& ch = c->chains[chain_id];
  if (ch.used) return fail(PP_ESTATE, "register_chain: chain %d already registered", chain_id);
  int st = PP_OK;
  if (!c->have[kSynth]) {
    // first synthetic chain: units that run synthetic frames and their buffers
    std::vector<Unit*> added;
    st = synth_alloc(&c->synth, kSynthUnits);
    for (int k = 0; k < kSynthUnits && !st; ++k) {
      Unit* u = new (std::nothrow) Unit();
      if (!u) { st = fail(PP_ENOMEM, "register_synthetic_chain: host allocation"); break; }
      u->precision = kSynth;
      added.push_back(u);
      st = cuda_status(cudaEventCreate(&u->start), "event");
      if (!st) st = cuda_status(cudaEventCreate(&u->done), "event");
    }
    if (st) {  // leave the context as it was
      for (Unit* u : added) {
        if (u->start) cudaEventDestroy(u->start);
        if (u->done) cudaEventDestroy(u->done);
        delete u;
      }
      synth_free(&c->synth);
      return st;
    }
    c->synth_first = (int)c->units.size();
    c->units.insert(c->units.end(), added.begin(), added.end());
    c->have[kSynth] = true;
    c->capacity[kSynth] = kMaxAdmitted;
  }
  const int ctas = synth_ctas(c->synth, util);
  int iters = 1;
  st = synth_calibrate(c->synth, ctas, kernel_us, c->aux, &iters);
  if (!st) st = chain_streams(c, &ch);
  if (st) return st;
  ch.used = true;
  ch.period_ms = period_ms;
  ch.deadline_ms = rel_deadline_ms;
  ch.precision = kSynth;
  ch.n_kernels = n_kernels;
  ch.kernel_us = kernel_us;
  ch.synth_ctas = ctas;
  ch.synth_iters = iters;
  ch.util = (double)ctas / c->synth.sms;
  return PP_OK;
}

int pp_submit_frames(pp_ctx* c, int32_t n, const int32_t* chain_ids, const float* const* xyzr,
                     const int64_t* n_points, int32_t is_device_ptr, double t_arrival_us,
                     const double* abs_deadline_us, uint64_t* frame_ids_out, int32_t* n_admitted) {
  return pp_submit_frames_ex(c, n, chain_ids, xyzr, n_points, is_device_ptr, t_arrival_us, abs_deadline_us,
                             nullptr, frame_ids_out, n_admitted);
}

size_t pp_result_bytes(pp_ctx* c, int32_t precision) {
  if (!c || (precision != PP_F32 && precision != PP_BF16) || !c->have[precision]) return 0;
  return c->models[precision].final_bytes();
}

int pp_submit_frames_ex(pp_ctx* c, int32_t n, const int32_t* chain_ids, const float* const* xyzr,
                        const int64_t* n_points, int32_t is_device_ptr, double t_arrival_us,
                        const double* abs_deadline_us, void* const* host_out, uint64_t* frame_ids_out,
                        int32_t* n_admitted) {
  if (n_admitted) *n_admitted = 0;
  if (!c || n < 1 || n > kMaxSubmit || !chain_ids || !xyzr || !n_points)
    return fail(PP_EINVAL, "submit: bad argument (n 1..%d, non-NULL arrays)", kMaxSubmit);
  if (is_device_ptr < PP_POINTS_HOST || is_device_ptr > PP_POINTS_PINNED)
    return fail(PP_EINVAL, "submit: is_device_ptr must be PP_POINTS_HOST, _DEVICE or _PINNED");
  const float* mapped[kMaxSubmit];  // what the kernels read: the device view of each frame
  for (int i = 0; i < n; ++i) {
    if (chain_ids[i] < 0 || chain_ids[i] >= PP_MAX_CHAINS) return fail(PP_EINVAL, "submit: bad chain");
    if (n_points[i] < 0 || n_points[i] > c->cfg.cap_points || (n_points[i] > 0 && !xyzr[i]))
      return fail(PP_EINVAL, "submit: n_points outside [0, cap_points] or NULL points");
    if (is_device_ptr && (reinterpret_cast<uintptr_t>(xyzr[i]) & 15u))
      return fail(PP_EINVAL, "submit: device or pinned points must be 16-byte aligned");
    mapped[i] = xyzr[i];
    if (is_device_ptr == PP_POINTS_PINNED && n_points[i] > 0) {
      cudaPointerAttributes at;
      if (cudaPointerGetAttributes(&at, xyzr[i]) != cudaSuccess || at.type != cudaMemoryTypeHost ||
          !at.devicePointer) {
        cudaGetLastError();
        return fail(PP_EINVAL, "submit: frame %d is not page-locked host memory", i);
      }
      mapped[i] = static_cast<const float*>(at.devicePointer);
    }
  }
  char* hout[kMaxSubmit] = {nullptr};  // device views of the host output buffers
  for (int i = 0; host_out && i < n; ++i) {
    if (!host_out[i]) continue;
    cudaPointerAttributes at;
    if ((reinterpret_cast<uintptr_t>(host_out[i]) & 15u) || cudaPointerGetAttributes(&at, host_out[i]) != cudaSuccess ||
        at.type != cudaMemoryTypeHost || !at.devicePointer) {
      cudaGetLastError();
      return fail(PP_EINVAL, "submit: host output %d is not 16-byte aligned page-locked host memory", i);
    }
    hout[i] = static_cast<char*>(at.devicePointer);
  }
  Frame* fs[kMaxSubmit];
  int k = 0, st = PP_OK;
  std::unique_lock<std::mutex> lk(c->mu);
  for (int i = 0; i < n; ++i)
    if (!c->chains[chain_ids[i]].used) return fail(PP_ESTATE, "submit: chain %d not registered", chain_ids[i]);
  // reserve, in order, a result slot (and a staging slot for host points) per frame
  for (; k < n; ++k) {
    const Chain& ch = c->chains[chain_ids[k]];
    const int p = ch.precision;
    const bool synth = p == kSynth;  // no points, no result slot, no staging
    if (c->admitted[p] >= c->capacity[p] || (!synth && c->pool[p].free.empty()) ||
        (!synth && !is_device_ptr && c->staging_free.empty())) {
      c->rejected += n - k;
      st = fail(PP_EAGAIN, "submit: HBM budget full");
      break;
    }
    Frame* f = new (std::nothrow) Frame();
    if (!f) {
      st = fail(PP_ENOMEM, "submit: host allocation");
      break;
    }
    f->id = c->next_id++;
    if (c->cfg.est_noise > 0) f->est_scale = pp_noise_factor(c->cfg.noise_seed, f->id, c->cfg.est_noise);
    if (hout[k] && !synth) {
      f->hout_dev = hout[k];
      f->hout_host = host_out[k];
    }
    f->chain = chain_ids[k];
    f->precision = p;
    f->t_arr = t_arrival_us;
    const double dl = abs_deadline_us ? abs_deadline_us[k] : 0.0;
    f->deadline = dl > 0 ? dl : t_arrival_us + ch.deadline_ms * 1000.0;
    f->n = synth ? 0 : n_points[k];
    c->admitted[p]++;
    if (synth) {
      fs[k] = f;
      continue;
    }
    f->rslot = c->pool[p].free.back();
    c->pool[p].free.pop_back();
    if (is_device_ptr) {
      f->src = mapped[k];  // read in place by the unit's kernels
      f->pinned = is_device_ptr == PP_POINTS_PINNED;
    } else {
      f->staging = c->staging_free.back();
      c->staging_free.pop_back();
      f->src = c->staging[f->staging];
    }
    fs[k] = f;
  }
  if (!is_device_ptr && k > 0) {
    lk.unlock();  // the copies run outside the lock; the slots are already ours
    for (int i = 0; i < k; ++i)
      if (fs[i]->n > 0) memcpy(const_cast<float*>(fs[i]->src), xyzr[i], (size_t)fs[i]->n * 16);
    lk.lock();
  }
  // the admitted frames become ready together, so one decision can batch all of them
  for (int i = 0; i < k; ++i) {
    Frame* f = fs[i];
    c->submitted++;
    if (c->first_arr < 0 || f->t_arr < c->first_arr) c->first_arr = f->t_arr;
    c->frames[f->id] = f;
    c->ready.push_back(f);
    if (frame_ids_out) frame_ids_out[i] = f->id;
  }
  if (n_admitted) *n_admitted = k;
  lk.unlock();
  if (k > 0) c->cv_work.notify_one();
  return st;
}

int pp_submit_frame(pp_ctx* c, int32_t chain_id, const float* xyzr, int64_t n_points,
                    int32_t is_device_ptr, double t_arrival_us, double abs_deadline_us,
                    uint64_t* frame_id_out) {
  return pp_submit_frames(c, 1, &chain_id, &xyzr, &n_points, is_device_ptr, t_arrival_us,
                          &abs_deadline_us, frame_id_out, nullptr);
}

int pp_poll(pp_ctx* c, pp_result* out, int32_t max, int32_t* n_out, int64_t timeout_us) {
  if (!c || !out || max <= 0 || !n_out) return fail(PP_EINVAL, "poll: bad argument");
  std::unique_lock<std::mutex> lk(c->mu);
  if (c->completed.empty() && timeout_us > 0)
    c->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [c] { return !c->completed.empty(); });
  int n = 0;
  while (n < max && !c->completed.empty()) {
    out[n] = c->completed.front();
    c->completed.pop_front();
    auto it = c->frames.find(out[n].frame_id);
    if (it != c->frames.end()) it->second->polled = true;
    ++n;
  }
  *n_out = n;
  return PP_OK;  // a failed unit's frames carry PP_FRAME_ERROR; pp_stats counts the failures
}

int pp_result_release_many(pp_ctx* c, int32_t n, const uint64_t* frame_ids) {
  if (!c || n < 0 || (n > 0 && !frame_ids)) return fail(PP_EINVAL, "release: bad argument");
  std::unique_lock<std::mutex> lk(c->mu);
  int st = PP_OK;
  for (int i = 0; i < n; ++i) {
    auto it = c->frames.find(frame_ids[i]);
    if (it == c->frames.end()) {
      st = fail(PP_EINVAL, "release: unknown frame %llu", (unsigned long long)frame_ids[i]);
      continue;
    }
    Frame* f = it->second;
    if (!f->done) {
      st = fail(PP_ESTATE, "release: frame %llu not completed", (unsigned long long)frame_ids[i]);
      continue;
    }
    if (!f->dropped) {
      free_result(c, f);
      c->admitted[f->precision]--;
    }
    c->frames.erase(it);
    delete f;
  }
  lk.unlock();
  c->cv_work.notify_one();
  return st;
}

int pp_result_release(pp_ctx* c, uint64_t frame_id) {
  if (!c) return fail(PP_EINVAL, "release: NULL context");
  return pp_result_release_many(c, 1, &frame_id);
}

int pp_get_stats(pp_ctx* c, pp_stats* s) {
  if (!c || !s) return fail(PP_EINVAL, "stats: NULL argument");
  std::lock_guard<std::mutex> lk(c->mu);
  memset(s, 0, sizeof(*s));
  s->submitted = c->submitted;
  s->done = c->n_done;
  s->dropped = c->n_dropped;
  s->missed = c->n_missed;
  s->rejected = c->rejected;
  double sum = 0;
  int nch = 0;
  for (int i = 0; i < PP_MAX_CHAINS; ++i) {
    const Chain& ch = c->chains[i];
    s->chain_frames[i] = ch.frames;
    s->chain_missed[i] = ch.missed;
    if (ch.frames) {
      sum += (double)ch.missed / (double)ch.frames;
      ++nch;
      std::vector<double> v = ch.lat;
      if (!v.empty()) {
        std::sort(v.begin(), v.end());
        s->chain_p99_us[i] = v[(size_t)std::floor(0.99 * (double)(v.size() - 1))];
      }
    }
  }
  s->overall_miss_ratio = nch ? sum / nch : 0.0;
  if (!c->lat_all.empty()) {
    std::vector<double> v = c->lat_all;
    std::sort(v.begin(), v.end());
    s->lat_p50_us = v[(size_t)std::floor(0.50 * (double)(v.size() - 1))];
    s->lat_p99_us = v[(size_t)std::floor(0.99 * (double)(v.size() - 1))];
    double m = 0;
    for (double x : v) m += x;
    s->lat_mean_us = m / (double)v.size();
  }
  if (c->n_done && c->last_done > c->first_arr)
    s->frames_per_s = (double)c->n_done / ((c->last_done - c->first_arr) * 1e-6);
  s->units_launched = c->launched;
  s->mean_batch = c->launched ? (double)c->batch_frames / (double)c->launched : 0.0;
  s->delayed_releases = c->delayed;
  s->delayed_us = c->delayed_us;
  s->collisions = c->collisions;
  s->sched_us_per_decision = c->decisions ? c->sched_us / (double)c->decisions : 0.0;
  s->th_urgent = c->th;
  s->device_errors = c->device_errors;
  s->device_error_code = c->device_error_code;
  s->decisions = c->decisions;
  return PP_OK;
}

int pp_stats_reset(pp_ctx* c) {
  if (!c) return fail(PP_EINVAL, "stats_reset: NULL context");
  std::lock_guard<std::mutex> lk(c->mu);
  c->submitted = c->n_done = c->n_dropped = c->n_missed = c->rejected = c->launched = 0;
  c->batch_frames = c->delayed = c->collisions = c->decisions = 0;
  c->delayed_us = c->sched_us = 0;
  c->first_arr = c->last_done = -1;
  c->lat_all.clear();
  c->device_errors = 0;
  c->device_error_code = 0;
  for (Chain& ch : c->chains) {
    ch.frames = ch.missed = 0;
    ch.lat.clear();
  }
  return PP_OK;
}

int pp_decision_log(pp_ctx* c, pp_decision_record* recs, int32_t max_recs, pp_policy_frame* ready,
                    int64_t max_ready, pp_policy_active* active, int64_t max_active, uint64_t* drops,
                    int64_t max_drops, int32_t* n_recs, int64_t* n_ready, int64_t* n_active,
                    int64_t* n_drops) {
  if (!c) return fail(PP_EINVAL, "decision_log: NULL context");
  std::lock_guard<std::mutex> lk(c->mu);
  if (n_recs) *n_recs = (int32_t)c->log.size();
  if (n_ready) *n_ready = (int64_t)c->log_ready.size();
  if (n_active) *n_active = (int64_t)c->log_active.size();
  if (n_drops) *n_drops = (int64_t)c->log_drops.size();
  if (!recs) return PP_OK;
  if (max_recs < (int64_t)c->log.size() || max_ready < (int64_t)c->log_ready.size() ||
      max_active < (int64_t)c->log_active.size() || max_drops < (int64_t)c->log_drops.size() ||
      (!c->log_ready.empty() && !ready) || (!c->log_active.empty() && !active) ||
      (!c->log_drops.empty() && !drops))
    return fail(PP_EINVAL, "decision_log: arrays smaller than the log");
  std::copy(c->log.begin(), c->log.end(), recs);
  std::copy(c->log_ready.begin(), c->log_ready.end(), ready);
  std::copy(c->log_active.begin(), c->log_active.end(), active);
  std::copy(c->log_drops.begin(), c->log_drops.end(), drops);
  return PP_OK;
}

int pp_destroy(pp_ctx* c) {
  if (!c) return PP_OK;
  c->stop.store(true);
  c->cv_work.notify_all();
  if (c->dispatcher.joinable()) c->dispatcher.join();
  const double t0 = now_us();
  bool busy = true;
  while (busy && now_us() - t0 < 10e6) {
    busy = false;
    for (Unit* u : c->units)
      if (u->running && cudaEventQuery(u->done) == cudaErrorNotReady) busy = true;
    if (busy) std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  cudaGetLastError();
  if (busy) return fail(PP_ETIMEDOUT, "destroy: units still running after 10 s");
  // every unit's completion event has fired; what may remain is the host notification queued
  // after it on the notify stream, which touches this context: let it finish first
  if (c->notify) cudaStreamSynchronize(c->notify);
  for (auto& ch : c->chains)
    for (cudaStream_t s : ch.streams) cudaStreamSynchronize(s);
  cudaGetLastError();
  destroy_units(c);
  delete c;
  return PP_OK;
}

int pp_replay(pp_ctx* c, const pp_arrival* arr, int64_t n, const float* const* clouds,
              const int64_t* cloud_points, int32_t n_clouds, int32_t is_device_ptr, double timeout_us,
              pp_replay_stats* out) {
  if (!c || !out || n < 0 || (n > 0 && (!arr || !clouds || !cloud_points)) || n_clouds <= 0 || timeout_us <= 0)
    return fail(PP_EINVAL, "replay: bad argument");
  for (int64_t k = 0; k < n; ++k) {
    if (k && arr[k].t_us < arr[k - 1].t_us) return fail(PP_EINVAL, "replay: arrivals not sorted by time");
    if (arr[k].cloud < 0 || arr[k].cloud >= n_clouds || arr[k].n_points < 0 ||
        arr[k].n_points > cloud_points[arr[k].cloud] || arr[k].chain_id < 0 || arr[k].chain_id >= PP_MAX_CHAINS)
      return fail(PP_EINVAL, "replay: arrival %lld names a bad chain, cloud or point count", (long long)k);
  }
  memset(out, 0, sizeof(*out));
  const double t0 = now_us();
  int64_t k = 0, outstanding = 0;
  double late_sum = 0;
  pp_result res[256];
  uint64_t ids[256];
  int st = PP_OK;
  while (k < n || outstanding > 0) {
    double t = now_us();
    while (k < n && t0 + arr[k].t_us <= t) {
      const pp_arrival& a = arr[k];
      const double due = t0 + a.t_us;
      const int rc = pp_submit_frame(c, a.chain_id, clouds[a.cloud], a.n_points, is_device_ptr, due, 0.0, nullptr);
      if (rc == PP_OK) {
        ++outstanding;
        ++out->submitted;
      } else if (rc == PP_EAGAIN) {
        ++out->rejected;
        ++out->chain_rejected[a.chain_id];
      } else {
        return rc;
      }
      const double late = now_us() - due;
      late_sum += late;
      out->submit_late_us_max = std::max(out->submit_late_us_max, late);
      ++k;
      t = now_us();
    }
    // wait for completions, but not past the next arrival
    double wait = 200.0;
    if (k < n) wait = std::min(wait, std::max(0.0, t0 + arr[k].t_us - now_us()));
    int32_t got = 0;
    st = pp_poll(c, res, 256, &got, (int64_t)wait);
    for (int i = 0; i < got; ++i) {
      ids[i] = res[i].frame_id;
      if (res[i].status == PP_FRAME_DROPPED) ++out->dropped;
      else ++out->completed;
    }
    if (got) pp_result_release_many(c, got, ids);
    outstanding -= got;
    if (st != PP_OK) break;
    if (k == n && outstanding > 0 && now_us() - (t0 + (n ? arr[n - 1].t_us : 0.0)) > timeout_us) {
      st = fail(PP_ETIMEDOUT, "replay: %lld frames still in flight %.0f us after the last arrival",
                (long long)outstanding, timeout_us);
      break;
    }
  }
  out->wall_s = (now_us() - t0) * 1e-6;
  out->submit_late_us_mean = n ? late_sum / (double)n : 0.0;
  return st;
}

}  // extern "C"
