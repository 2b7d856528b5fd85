"""Oracle of the urgency-aware release policy -- TEST INFRASTRUCTURE ONLY (see ``oracle``).

Restates, in plain Python, the paper's scheduling rules as this library applies them to whole
release units (a unit = up to ``max_batch`` frames run as one launch):

* urgency (Eq. 2): UL(t) = 1 / (t_arr + D - sum of remaining GPU estimates - sum of remaining
  CPU estimates - t).  With slack = t_arr + D - rem_gpu - rem_cpu - t, UL = 1/slack for
  slack > 0; a frame with slack <= 0 is treated as least urgent (UL = -inf);
* early chain exit (Section 4.3): a frame whose urgency is negative (slack < 0) when its next
  unit would start is dropped;
* CPU-priority ranking (Section 4.3, Table 2): descending urgency, ties by lower chain id;
* task-level stream binding with reservation (Section 4.4.3): level 0 (highest stream
  priority) is reserved for UL > TH_urgent; other units get their urgency rank among the
  non-urgent active units normalised onto levels 1 .. NUM_PRI-1;
* delayed launching (Section 4.4.4): a unit is held while another chain's active unit has
  UL > TH_urgent and a higher urgency than it; units with utilisation below the exemption
  threshold are never held;
* batched launch synchronisation with overlap (Section 4.4.5): launches accumulate into a batch
  until the sum of their estimated GPU times reaches Delta_eval; the batch then closes, and no
  further launch happens while ``max_closed`` closed batches are unfinished (2 = overlapped:
  wait for the previous batch; 1 = synchronous batched; 0 = no synchronisation);
* the overall deadline-miss ratio (Eq. 3): mean over chains of each chain's miss ratio;
* urgency-centric CPU scheduling (Section 4.3), in the DES only: CPU segments that follow a
  chain's GPU units run on a few cores either in order of readiness (the default scheduler's
  view) or preemptively by descending urgency, re-ranked at every event.

The comparison policies of the paper's Section 6.4 (EDF, SJF, HRRN and lowest chain utilisation
first; the paper names them without definitions) are the textbook orders: a priority value
replaces the urgency in ordering frames and ranking active units onto stream levels
0 .. NUM_PRI-1, without early exit, reservation or delaying:

* EDF: earliest absolute deadline first (priority -deadline);
* SJF: shortest remaining estimate e = est_gpu + est_cpu first (priority -e);
* HRRN: highest response ratio (waited + e) / e first (+inf for e <= 0);
* LCUF: lowest chain utilisation e / period first (priority -e / period; -inf without a period);
* SAEDF (slack-aware EDF; reading): earliest deadline first among frames whose slack is still
  >= 0, every frame with negative slack after them, again by deadline (priority -deadline, less
  10^15 us for a negative slack);
* EQDF (earliest quasi-deadline first; reading): priority -(deadline - lambda e), lambda =
  ``eqdf_lambda`` (0 gives EDF; 1 orders by latest start time, like the urgency order).

Readings where the paper is silent: urgency order breaks ties by
(chain id, arrival time, frame id); the FIFO baseline orders by (arrival, chain id, frame id);
rank r counts the active non-urgent units strictly more urgent than the candidate, n counts
them plus the candidate, level = 1 + floor(r (NUM_PRI-1) / n); the delay rule compares against
*other* chains only (two urgent chains would otherwise hold each other forever); a dropped frame
counts as a miss.
"""
from __future__ import annotations

import dataclasses
import heapq
import math
from typing import Callable, Dict, List, Optional, Sequence, Tuple

POLICY_FIFO = 0
POLICY_URGENCY = 1
POLICY_EDF = 2
POLICY_SJF = 3
POLICY_HRRN = 4
POLICY_LCUF = 5
POLICY_SAEDF = 6
POLICY_EQDF = 7

NONE, RELEASE, WAIT, DELAY = 0, 1, 2, 3


@dataclasses.dataclass
class PolicyConfig:
    policy: int = POLICY_URGENCY
    max_batch: int = 8
    delta_eval_us: float = 500.0
    max_closed: int = 2
    th_urgent: float = 0.0          # 1/us; <= 0 disables reservation and delaying
    util_exempt: float = 0.1
    early_exit: bool = True
    num_pri: int = 6
    eqdf_lambda: float = 0.5        # EQDF: quasi-deadline = deadline - lambda x estimate


@dataclasses.dataclass
class Ready:
    frame_id: int
    chain_id: int
    t_arr: float
    deadline: float                 # absolute: t_arr + D
    est_gpu: float                  # remaining GPU estimate (us)
    est_cpu: float = 0.0            # remaining CPU estimate (us)
    precision: int = 0
    util: float = 1.0
    period: float = 0.0             # the chain's period (us), for LCUF


@dataclasses.dataclass
class Active:
    chain_id: int
    ul: float                       # priority (urgency for the urgency policy) at release


@dataclasses.dataclass
class Decision:
    kind: int
    frames: List[int]
    level: int
    drops: List[int]


def slack(f: Ready, t: float) -> float:
    """Denominator of Eq. 2: t_arr + D - remaining GPU - remaining CPU - t."""
    return f.deadline - f.est_gpu - f.est_cpu - t


def urgency(s: float) -> float:
    """Eq. 2 from a slack value; non-positive slack is least urgent."""
    return 1.0 / s if s > 0 else -math.inf


def table2_urgency(D: float, e_cpu: float, e_gpu: float) -> float:
    """Eq. 2 at t = t_arr with all work of the chain remaining (how Table 2 is computed)."""
    return 1.0 / (D - e_cpu - e_gpu)


def priority_ranks(uls: Sequence[float]) -> List[int]:
    """Section 4.3: rank chains by descending urgency; the most urgent gets PRI 1.
    Ties go to the lower chain id (list position)."""
    order = sorted(range(len(uls)), key=lambda i: (-uls[i], i))
    pri = [0] * len(uls)
    for r, i in enumerate(order):
        pri[i] = r + 1
    return pri


def stream_level(ul: float, active: Sequence[Active], cfg: PolicyConfig) -> int:
    """Section 4.4.3: reserved top level for UL > TH_urgent, else normalised rank."""
    if cfg.num_pri <= 1:
        return 0
    if cfg.th_urgent > 0 and ul > cfg.th_urgent:
        return 0
    nonurg = [a.ul for a in active if not (cfg.th_urgent > 0 and a.ul > cfg.th_urgent)]
    r = sum(1 for u in nonurg if u > ul)
    n = len(nonurg) + 1
    return 1 + (r * (cfg.num_pri - 1)) // n


def must_delay(f: Ready, ul: float, active: Sequence[Active], cfg: PolicyConfig) -> bool:
    """Section 4.4.4 delay test for the unit headed by ``f``."""
    if cfg.policy != POLICY_URGENCY or cfg.th_urgent <= 0 or f.util < cfg.util_exempt:
        return False
    return any(a.chain_id != f.chain_id and a.ul > cfg.th_urgent and a.ul > ul for a in active)


def priority(f: Ready, t: float, cfg: PolicyConfig) -> float:
    """The value a policy releases by (higher first) and ranks active units by."""
    e = f.est_gpu + f.est_cpu
    if cfg.policy == POLICY_URGENCY:
        return urgency(slack(f, t))
    if cfg.policy == POLICY_EDF:
        return -f.deadline
    if cfg.policy == POLICY_SJF:
        return -e
    if cfg.policy == POLICY_HRRN:
        return (t - f.t_arr + e) / e if e > 0 else math.inf
    if cfg.policy == POLICY_LCUF:
        return -(e / f.period) if f.period > 0 else -math.inf
    if cfg.policy == POLICY_SAEDF:
        # earliest deadline among frames that can still meet theirs, then the rest: the
        # second group is pushed back by a constant far larger than any deadline
        return -f.deadline - (1e15 if slack(f, t) < 0 else 0.0)
    if cfg.policy == POLICY_EQDF:
        return -(f.deadline - cfg.eqdf_lambda * e)
    return -f.t_arr


def order_key(f: Ready, t: float, cfg: PolicyConfig) -> tuple:
    if cfg.policy == POLICY_URGENCY:
        return (slack(f, t), f.chain_id, f.t_arr, f.frame_id)
    if cfg.policy == POLICY_FIFO:
        return (f.t_arr, f.chain_id, f.frame_id)
    return (-priority(f, t, cfg), f.chain_id, f.t_arr, f.frame_id)


def rank_level(p: float, active: Sequence[Active], num_pri: int) -> int:
    """Comparison policies: the candidate's rank among all active units (strictly higher
    priority first) spread over levels 0 .. NUM_PRI-1."""
    if num_pri <= 1:
        return 0
    r = sum(1 for a in active if a.ul > p)
    return (r * num_pri) // (len(active) + 1)


def decide(t: float, ready: Sequence[Ready], active: Sequence[Active], closed_pending: int,
           cfg: PolicyConfig) -> Decision:
    """One release decision at time t (all times in microseconds)."""
    drops: List[int] = []
    cand = list(ready)
    if cfg.policy == POLICY_URGENCY and cfg.early_exit:
        drops = [f.frame_id for f in cand if slack(f, t) < 0]
        cand = [f for f in cand if slack(f, t) >= 0]
    if not cand:
        return Decision(NONE, [], 0, drops)
    if cfg.max_closed > 0 and closed_pending >= cfg.max_closed:
        return Decision(WAIT, [], 0, drops)
    cand.sort(key=lambda f: order_key(f, t, cfg))
    head = cand[0]
    ul = urgency(slack(head, t))
    if must_delay(head, ul, active, cfg):
        return Decision(DELAY, [], 0, drops)
    batch = [head.frame_id]
    for f in cand[1:]:
        if len(batch) >= max(1, cfg.max_batch):
            break
        if f.precision == head.precision:
            batch.append(f.frame_id)
    if cfg.policy == POLICY_URGENCY:
        level = stream_level(ul, active, cfg)
    elif cfg.policy == POLICY_FIFO:
        level = max(0, cfg.num_pri - 1)
    else:
        level = rank_level(priority(head, t, cfg), active, cfg.num_pri)
    return Decision(RELEASE, batch, level, drops)


class BatchGate:
    """Section 4.4.5 bookkeeping: open-batch sum, closed batches still running."""

    def __init__(self, delta_eval_us: float):
        self.delta = delta_eval_us
        self.open_sum = 0.0
        self.open_units: List[int] = []
        self.closed: List[List[int]] = []      # unit ids per closed, unfinished batch

    def launched(self, unit_id: int, est_us: float) -> bool:
        """Adds a launched unit; returns True when this launch closes the batch."""
        self.open_units.append(unit_id)
        self.open_sum += est_us
        if self.open_sum >= self.delta:
            self.closed.append(self.open_units)
            self.open_units, self.open_sum = [], 0.0
            return True
        return False

    def finished(self, unit_id: int) -> None:
        """A unit completed; closed batches complete in launch order (one stream of events)."""
        for b in self.closed:
            if unit_id in b:
                b.remove(unit_id)
        while self.closed and not self.closed[0]:
            self.closed.pop(0)
        if unit_id in self.open_units:
            self.open_units.remove(unit_id)

    @property
    def pending(self) -> int:
        return sum(1 for b in self.closed if b)


def batch_boundaries(estimates: Sequence[float], delta_eval: float) -> List[int]:
    """Indices after which a synchronisation point is inserted (Section 4.4.5): kernels are
    added to the open batch, which closes once the sum of its estimates reaches Delta_eval."""
    out, s = [], 0.0
    for i, e in enumerate(estimates):
        s += e
        if s >= delta_eval:
            out.append(i)
            s = 0.0
    return out


def overall_miss_ratio(per_chain: Dict[int, Tuple[int, int]]) -> float:
    """Eq. 3: (1/N) * sum over chains of misses / total.  ``per_chain[c] = (misses, total)``;
    chains with no frames are skipped."""
    vals = [m / n for (m, n) in per_chain.values() if n > 0]
    return sum(vals) / len(vals) if vals else 0.0


@dataclasses.dataclass
class SimFrame:
    frame_id: int
    chain_id: int
    t_arr: float
    deadline: float
    stages: List[float]             # true GPU durations per unit (us)
    precision: int = 0
    util: float = 1.0
    est: Optional[List[float]] = None   # estimates per unit (defaults to the true durations)
    period: float = 0.0                 # the chain's period (us), for LCUF
    cpu: Optional[List[float]] = None   # CPU segment after each GPU unit (us; 0 = none)


@dataclasses.dataclass
class SimResult:
    releases: List[Tuple[float, List[Tuple[int, int]], int]]   # (t, [(frame, stage)], level)
    done: Dict[int, float]            # frame -> completion time
    dropped: Dict[int, float]         # frame -> drop time
    missed: Dict[int, bool]


def simulate(frames: Sequence[SimFrame], cfg: PolicyConfig, delay_quantum_us: float = 1000.0,
             unit_time: Optional[Callable[[List[float]], float]] = None,
             servers: int = 1, cpu_cores: int = 1, cpu_policy: str = "fifo") -> SimResult:
    """Discrete-event simulation of the release policy.

    GPU model: ``servers`` identical non-preemptive servers; a released unit waits in a queue
    ordered by (stream level, release order) and runs for ``unit_time(stage durations of its
    frames)`` (default: the sum).  Decision points: frame arrival, unit completion, delay
    wake-up, CPU segment completion.  A frame re-enters the ready set after each of its units
    (and the CPU segment that follows it, if any) until all are done.

    CPU model (Section 4.3; frames with ``cpu`` segments): ``cpu_cores`` cores.  ``cpu_policy``
    "fifo": segments run in the order they became ready, to completion (the default fair
    scheduler's view of equal tasks).  "urgency": the paper's urgency-centric CPU scheduling --
    fixed real-time priorities by descending urgency: whenever a segment becomes ready or a core
    frees, the ready and running segments are ranked by their frames' urgency at that moment and
    the most urgent ones hold the cores, a less urgent running segment being preempted (its
    remaining time resumes later).  The GPU policy's slack counts the remaining CPU time (the
    true segment durations serve as the estimates).
    """
    if unit_time is None:
        unit_time = lambda ds: float(sum(ds))
    if cpu_policy not in ("fifo", "urgency"):
        raise ValueError("cpu_policy must be fifo or urgency")
    by_id = {f.frame_id: f for f in frames}
    est = {f.frame_id: (f.est if f.est is not None else list(f.stages)) for f in frames}
    cpu = {f.frame_id: (f.cpu if f.cpu is not None else [0.0] * len(f.stages)) for f in frames}
    nxt = {f.frame_id: 0 for f in frames}
    cpu_left: Dict[int, float] = {}                  # frame -> remaining time of its CPU segment
    cpu_ready: List[Tuple[float, int]] = []          # (ready time, frame), waiting for a core
    cpu_run: Dict[int, float] = {}                   # frame -> time its current run started
    arrivals = sorted(frames, key=lambda f: (f.t_arr, f.frame_id))
    ai = 0
    ready: Dict[int, SimFrame] = {}
    active: Dict[int, Tuple[Active, List[Tuple[int, int]], int]] = {}  # unit -> (akb, members, level)
    queue: List[Tuple[int, int, int]] = []           # (level, seq, unit)
    running: List[Tuple[float, int]] = []            # (t_end, unit) heap
    gate = BatchGate(cfg.delta_eval_us)
    wake: Optional[float] = None
    res = SimResult([], {}, {}, {})
    seq = 0
    t = 0.0

    def start_units(now: float) -> None:
        while queue and len(running) < servers:
            _, _, u = heapq.heappop(queue)
            _, members, _ = active[u]
            heapq.heappush(running, (now + unit_time([by_id[fid].stages[k] for fid, k in members]), u))

    def rem_cpu(fid: int) -> float:
        k = nxt[fid]
        return cpu_left.get(fid, 0.0) + sum(cpu[fid][k:])

    def slack_of(fid: int, now: float) -> float:
        f = by_id[fid]
        return f.deadline - sum(est[fid][nxt[fid]:]) - rem_cpu(fid) - now

    def schedule_cpu(now: float) -> None:
        # account the time run so far, then pick who holds the cores
        for fid, t0 in list(cpu_run.items()):
            cpu_left[fid] -= now - t0
            cpu_run[fid] = now
        if cpu_policy == "fifo":
            cpu_ready.sort()
            while cpu_ready and len(cpu_run) < cpu_cores:
                _, fid = cpu_ready.pop(0)
                cpu_run[fid] = now
            return
        # urgency: most urgent first (least slack; ties by chain id, arrival, frame id)
        cands = [fid for _, fid in cpu_ready] + list(cpu_run)
        cands.sort(key=lambda fid: (slack_of(fid, now), by_id[fid].chain_id, by_id[fid].t_arr, fid))
        hold = set(cands[:cpu_cores])
        for fid in list(cpu_run):
            if fid not in hold:  # preempted
                del cpu_run[fid]
                cpu_ready.append((now, fid))
        cpu_ready[:] = [(tr, fid) for tr, fid in cpu_ready if fid not in hold]
        for fid in hold:
            cpu_run.setdefault(fid, now)

    def next_cpu_end() -> Optional[Tuple[float, int]]:
        if not cpu_run:
            return None
        return min((t0 + cpu_left[fid], fid) for fid, t0 in cpu_run.items())

    def frame_stage_done(fid: int, now: float) -> None:
        f = by_id[fid]
        if nxt[fid] >= len(f.stages):
            res.done[fid] = now
            res.missed[fid] = now > f.deadline
        else:
            ready[fid] = f

    while True:
        # decisions at time t
        while True:
            rlist = [Ready(f.frame_id, f.chain_id, f.t_arr, f.deadline,
                           sum(est[f.frame_id][nxt[f.frame_id]:]), rem_cpu(f.frame_id), f.precision, f.util,
                           f.period)
                     for f in ready.values()]
            d = decide(t, rlist, [a for a, _, _ in active.values()], gate.pending, cfg)
            for fid in d.drops:
                res.dropped[fid] = t
                res.missed[fid] = True
                del ready[fid]
            if d.kind != RELEASE:
                if d.kind == DELAY:
                    wake = t + delay_quantum_us if wake is None else wake
                break
            members = [(fid, nxt[fid]) for fid in d.frames]
            head = by_id[d.frames[0]]
            ul = priority(Ready(head.frame_id, head.chain_id, head.t_arr, head.deadline,
                                sum(est[head.frame_id][nxt[head.frame_id]:]), rem_cpu(head.frame_id),
                                head.precision, head.util, head.period), t, cfg)
            unit = seq
            seq += 1
            active[unit] = (Active(head.chain_id, ul), members, d.level)
            for fid in d.frames:
                del ready[fid]
            res.releases.append((t, members, d.level))
            gate.launched(unit, sum(est[fid][k] for fid, k in members))
            heapq.heappush(queue, (d.level, unit, unit))
        start_units(t)
        # next event
        cands = []
        if ai < len(arrivals):
            cands.append(arrivals[ai].t_arr)
        if running:
            cands.append(running[0][0])
        if wake is not None:
            cands.append(wake)
        ce = next_cpu_end()
        if ce is not None:
            cands.append(ce[0])
        if not cands:
            break
        t = max(t, min(cands))
        if wake is not None and wake <= t:
            wake = None
        cpu_changed = False
        while True:  # CPU segments ending by t (in end order)
            ce = next_cpu_end()
            if ce is None or ce[0] > t:
                break
            fid = ce[1]
            del cpu_run[fid]
            del cpu_left[fid]
            frame_stage_done(fid, ce[0])
            cpu_changed = True
        while running and running[0][0] <= t:
            _, u = heapq.heappop(running)
            _, members, _ = active.pop(u)
            gate.finished(u)
            for fid, k in members:
                nxt[fid] = k + 1
                seg = cpu[fid][k]
                if seg > 0:  # the CPU part that follows this GPU unit
                    cpu_left[fid] = seg
                    cpu_ready.append((t, fid))
                    cpu_changed = True
                else:
                    frame_stage_done(fid, t)
            start_units(t)
        if cpu_changed or cpu_run or cpu_ready:
            schedule_cpu(t)
        while ai < len(arrivals) and arrivals[ai].t_arr <= t:
            ready[arrivals[ai].frame_id] = arrivals[ai]
            ai += 1
    return res


def miss_ratio_of(res: SimResult, frames: Sequence[SimFrame]) -> float:
    per: Dict[int, List[int]] = {}
    for f in frames:
        m, n = per.get(f.chain_id, [0, 0])
        per[f.chain_id] = [m + int(res.missed.get(f.frame_id, True)), n + 1]
    return overall_miss_ratio({c: (m, n) for c, (m, n) in per.items()})
