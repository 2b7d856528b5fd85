// The release rule as a pure function of (time, ready frames, active units, closed batches).
//
// Urgency (Eq. 2): UL = 1 / slack with slack = deadline - remaining GPU estimate - remaining
// CPU estimate - t; non-positive slack is least urgent.  Early chain exit (Section 4.3): frames
// with negative slack are dropped.  Batched synchronisation (Section 4.4.5): no release while
// `max_closed` closed batches are unfinished.  Order: least slack first (ties: chain id,
// arrival, frame id); FIFO baseline: arrival, chain id, frame id.  Delayed launching
// (Section 4.4.4): hold the head while another chain's active unit is above TH_urgent and more
// urgent, unless the head's utilisation is below the exemption threshold.  Stream binding with
// reservation (Section 4.4.3): level 0 for UL > TH_urgent; otherwise the urgency rank among the
// non-urgent active units, normalised onto levels 1..NUM_PRI-1.  Frames of the head's precision
// fill the unit up to max_batch, in order.  The comparison policies (EDF, SJF, HRRN, LCUF,
// SAEDF, EQDF) only change the priority that orders frames and ranks active units (levels
// 0..NUM_PRI-1, no reservation, no delaying, no early exit).
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "pp.h"

namespace {

double slack_of(const pp_policy_frame& f, double t) {
  return f.deadline_us - f.est_gpu_us - f.est_cpu_us - t;
}
double ul_of(double s) { return s > 0 ? 1.0 / s : -std::numeric_limits<double>::infinity(); }
bool urgent(double ul, const pp_policy_config& c) { return c.th_urgent > 0 && ul > c.th_urgent; }

double prio_of(const pp_policy_config& c, const pp_policy_frame& f, double t) {
  const double inf = std::numeric_limits<double>::infinity();
  const double e = f.est_gpu_us + f.est_cpu_us;
  switch (c.policy) {
    case PP_POLICY_URGENCY: return ul_of(slack_of(f, t));
    case PP_POLICY_EDF: return -f.deadline_us;
    case PP_POLICY_SJF: return -e;
    case PP_POLICY_HRRN: return e > 0 ? (t - f.t_arr_us + e) / e : inf;
    case PP_POLICY_LCUF: return f.period_us > 0 ? -(e / f.period_us) : -inf;
    // frames that can no longer make their deadline sort after every frame that can
    case PP_POLICY_SAEDF: return -f.deadline_us - (slack_of(f, t) < 0 ? 1e15 : 0.0);
    case PP_POLICY_EQDF: return -(f.deadline_us - c.eqdf_lambda * e);
    default: return -f.t_arr_us;
  }
}

}  // namespace

extern "C" double pp_policy_priority(const pp_policy_config* cfg, double t, const pp_policy_frame* f) {
  if (!cfg || !f) return -std::numeric_limits<double>::infinity();
  return prio_of(*cfg, *f, t);
}

extern "C" int pp_policy_decide(const pp_policy_config* cfg, double t, const pp_policy_frame* ready,
                                int32_t n_ready, const pp_policy_active* active, int32_t n_active,
                                int32_t closed_pending, pp_policy_decision* out, uint64_t* drops,
                                int32_t drops_cap) {
  if (!cfg || !out || n_ready < 0 || n_active < 0 || (n_ready && !ready) || (n_active && !active) ||
      cfg->policy < PP_POLICY_FIFO || cfg->policy > PP_POLICY_EQDF)
    return PP_EINVAL;
  const pp_policy_config& c = *cfg;
  out->kind = PP_DECIDE_NONE;
  out->level = 0;
  out->n_frames = 0;
  out->n_drops = 0;
  const bool urg = c.policy == PP_POLICY_URGENCY;
  std::vector<int> cand;
  cand.reserve(n_ready);
  for (int i = 0; i < n_ready; ++i) {
    if (urg && c.early_exit && slack_of(ready[i], t) < 0) {
      if (drops && out->n_drops < drops_cap) drops[out->n_drops] = ready[i].frame_id;
      ++out->n_drops;
    } else {
      cand.push_back(i);
    }
  }
  if (cand.empty()) return PP_OK;
  if (c.max_closed > 0 && closed_pending >= c.max_closed) {
    out->kind = PP_DECIDE_WAIT;
    return PP_OK;
  }
  const bool fifo = c.policy == PP_POLICY_FIFO;
  auto before = [&](int a, int b) {
    const pp_policy_frame& x = ready[a];
    const pp_policy_frame& y = ready[b];
    if (urg) {
      const double sx = slack_of(x, t), sy = slack_of(y, t);
      if (sx != sy) return sx < sy;
    } else if (fifo) {
      if (x.t_arr_us != y.t_arr_us) return x.t_arr_us < y.t_arr_us;
      if (x.chain_id != y.chain_id) return x.chain_id < y.chain_id;
      return x.frame_id < y.frame_id;
    } else {
      const double px = prio_of(c, x, t), py = prio_of(c, y, t);
      if (px != py) return px > py;
    }
    if (x.chain_id != y.chain_id) return x.chain_id < y.chain_id;
    if (x.t_arr_us != y.t_arr_us) return x.t_arr_us < y.t_arr_us;
    return x.frame_id < y.frame_id;
  };
  std::sort(cand.begin(), cand.end(), before);
  const pp_policy_frame& head = ready[cand[0]];
  const double ul = ul_of(slack_of(head, t));
  if (urg && c.th_urgent > 0 && head.util >= c.util_exempt) {
    for (int i = 0; i < n_active; ++i) {
      if (active[i].chain_id != head.chain_id && urgent(active[i].ul, c) && active[i].ul > ul) {
        out->kind = PP_DECIDE_DELAY;
        return PP_OK;
      }
    }
  }
  const int cap = std::max(1, std::min(c.max_batch, 8));
  out->frames[out->n_frames++] = head.frame_id;
  for (size_t k = 1; k < cand.size() && out->n_frames < cap; ++k)
    if (ready[cand[k]].precision == head.precision) out->frames[out->n_frames++] = ready[cand[k]].frame_id;
  if (fifo) {
    out->level = std::max(0, c.num_pri - 1);
  } else if (!urg) {
    // rank among the active units by the policy's priority, onto levels 0..NUM_PRI-1
    const double p = prio_of(c, head, t);
    int r = 0;
    for (int i = 0; i < n_active; ++i)
      if (active[i].ul > p) ++r;
    out->level = c.num_pri <= 1 ? 0 : (r * c.num_pri) / (n_active + 1);
  } else if (c.num_pri <= 1 || urgent(ul, c)) {
    out->level = 0;
  } else {
    int r = 0, n = 1;
    for (int i = 0; i < n_active; ++i) {
      if (urgent(active[i].ul, c)) continue;
      ++n;
      if (active[i].ul > ul) ++r;
    }
    out->level = 1 + (r * (c.num_pri - 1)) / n;
  }
  out->kind = PP_DECIDE_RELEASE;
  return PP_OK;
}
