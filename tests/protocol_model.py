"""Executable model of the synchronisation protocol of score_tc_kernel.

Test infrastructure (plain Python, no GPU).  The model mirrors, step for step,
the programs the warps of one CTA of the tensor-core scoring kernel run:

* the TMA warp, which fills a ring of NS coordinate-tile stages and two
  direction buffers;
* the GEMM1 warp, which for every tile g waits for the tile's stage and for
  D1 buffer g % ND (a ring of ND buffers in tensor memory) to be released,
  arrives on the buffer's barrier (which tells the rounding warps that the
  stage has landed) and issues the projections into the buffer (the barrier
  completes on that arrival plus the MMA's commit); it waits for each item's
  directions and commits their release after the item's last GEMM1;
* two GEMM2 warps (streams): GEMM2 warp v takes the tiles g with
  g % 2 == v and waits for A2-full barrier [g % NWG][v] (one per warpgroup
  and stream, so that each is waited for by one stream, phase after phase);
* NWG = ND rounding warpgroups (four warps each): warpgroup w = g % NWG owns
  D1 buffer w; it waits for D1 of tile g, loads D1 chunk by chunk, releases
  the buffer once the last chunk is in registers, reads the indicator
  magnitudes from the tile's stage chunk by chunk (the last ones after the
  release), rounds, and stores the indicator operand into its own A2 buffer;
* GEMM2 of tile g (MMA warp g % 2) reads A2[g % NWG] and accumulates into
  the stream's accumulator D2[v][p % NB2], p the index of the tile's
  accumulation period among stream v's periods (a period is at most F of the
  stream's tiles of one item);
* the fold warpgroup (four warps), which reads the accumulators at the end of
  each period -- per item, period i of stream 0, then period i of stream 1,
  for i = 0, 1, ... -- and releases them;
* the tcgen05 operations (MMAs and commits) of the issuing warps, which
  execute in issue order per warp and in any order across the warps; a commit
  arrives on its mbarrier once every earlier operation of its warp has
  executed;
* the TMA copies, which complete in any order;
* the mbarriers (arrival count, transaction bytes, completed phases) with
  their parity waits.

A seeded random scheduler runs one enabled agent at a time (a warp, the head
of an MMA queue, a pending copy).  The checker raises ProtocolError on

* a deadlock: nothing can run and some warp has not finished;
* a parity wait that could alias: a warp waits for phase k of a barrier that
  has already completed phase k + 1, or that has not yet completed phase
  k - 1 (mbarrier.try_wait.parity cannot tell phase k from phase k + 2, so
  such a wait would block, or pass, on the wrong phase);
* an arrival that would count towards the wrong phase (more arrivals than
  the barrier's count while a phase is open is caught as a phase completing
  early, which the data checks then see);
* a data hazard: an operand read before the data it needs was written (D1 of
  the wrong tile, a stage or direction buffer not yet landed, A2 or D2
  holding the wrong tiles), or a buffer overwritten before its last reader
  has consumed it.

`fail_prob` > 0 also exercises the failure path: a wait that is not yet
satisfied may give up (a bounded wait running out), exactly as the kernel's
waits do; the warp then sets the CTA's abort flag, which makes every other
unsatisfied wait give up at once, and leaves its loop.  The checker then also
requires that no MMA or copy is outstanding when the last warp reaches the
teardown (TMEM is freed and the CTA exits there).

`mutation` plants one known mistake in the protocol (the checker must catch
it): "refill_early" refills a stage one tile too soon, "no_a2_wait" stores A2
without waiting for the GEMM2 that read it last, "no_d1_wait" issues GEMM1
without waiting for the D1 buffer to be released, "release_early" releases D1
before loading it, "no_d2_wait" starts a period without waiting for the fold
of the period that used the accumulator before, "no_drain" lets the GEMM1
warp skip its drain.
"""
from __future__ import annotations

import random


class ProtocolError(AssertionError):
    pass


class Barrier:
    """An mbarrier: `count` arrivals plus transaction bytes complete a phase."""

    def __init__(self, name, count=1):
        self.name = name
        self.count = count
        self.pending = count
        self.tx = 0
        self.done = 0  # completed phases
        self.waiters = {}  # warp -> awaited phase

    def _check_complete(self):
        if self.pending == 0 and self.tx == 0:
            self.done += 1
            self.pending = self.count
            for w, k in self.waiters.items():
                if self.done >= k + 2:
                    raise ProtocolError("%s: %s waits for phase %d, but phase %d has completed too"
                                        % (self.name, w, k, k + 1))

    def arrive(self):
        self.pending -= 1
        if self.pending < 0:
            raise ProtocolError("%s: more arrivals than its count" % self.name)
        self._check_complete()

    def expect_tx(self, nbytes):
        self.tx += nbytes

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        self._check_complete()

    def start_wait(self, who, k):
        if self.done >= k + 2:
            raise ProtocolError("%s: %s starts waiting for phase %d after phase %d completed"
                                % (self.name, who, k, k + 1))
        if self.done < k:
            # the barrier is still in phase k - 1 (or earlier), whose parity is
            # not k's: a parity wait for phase k would pass at once
            raise ProtocolError("%s: %s waits for phase %d while phase %d has not completed"
                                % (self.name, who, k, k - 1))
        self.waiters[who] = k

    def ready(self, k):
        return self.done >= k + 1

    def end_wait(self, who):
        self.waiters.pop(who, None)


def make_items(rng, n_items, max_tiles):
    return [rng.randint(1, max_tiles) for _ in range(n_items)]


class Cta:
    """One CTA of the kernel; `items` is the number of tiles of each item."""

    def __init__(self, items, ns, nd, flush, seed, mutation=None, fail_prob=0.0, async_weight=1.0,
                 slow_mma=False, nwg=3, nb2=1):
        self.rng = random.Random(seed)
        self.async_weight = async_weight  # < 1: MMAs and copies lag behind the warps
        self.slow_mma = slow_mma  # the GEMM1 warp's MMAs far slower than everything else
        self.fail_prob = fail_prob
        self.abort = False
        self.ns = ns
        self.nd = nd
        self.F = flush
        # each rounding warpgroup owns one D1 buffer (so that its barrier is
        # waited for by one warpgroup, phase after phase): as many
        # warpgroups as buffers
        self.nwg = nwg = nd
        self.nb2 = nb2
        self.mut = mutation
        self.items = list(items)
        # the CTA's tile sequence: (item, j, ntile)
        self.tiles = [(i, j, nt) for i, nt in enumerate(items) for j in range(nt)]
        self.T = len(self.tiles)
        self.n_items = len(items)
        # accumulation periods of each GEMM2 stream: its tiles of an item, F at
        # a time; tile -> (stream, period), first / last tile of a period
        self.period_of = {}
        self.period_tiles = {}
        self.first = {}
        self.last = {}
        self.item_periods = []  # per item: [periods of stream 0, periods of stream 1]
        pcount = [0, 0]
        g = 0
        for i, nt in enumerate(items):
            own = [[g + j for j in range(nt) if (g + j) % 2 == w] for w in range(2)]
            per_item = [[], []]
            for w in range(2):
                for a in range(0, len(own[w]), flush):
                    chunk = own[w][a:a + flush]
                    p = pcount[w]
                    pcount[w] += 1
                    per_item[w].append(p)
                    self.period_tiles[(w, p)] = set(chunk)
                    for t in chunk:
                        self.period_of[t] = (w, p)
                        self.first[t] = t == chunk[0]
                        self.last[t] = t == chunk[-1]
            self.item_periods.append(per_item)
            g += nt
        # barriers
        self.sfull = [Barrier("sfull[%d]" % s) for s in range(ns)]
        self.sempty = [Barrier("sempty[%d]" % s) for s in range(ns)]
        self.dfull = [Barrier("dfull[%d]" % b) for b in range(2)]
        self.dempty = [Barrier("dempty[%d]" % b) for b in range(2)]
        self.d1full = [Barrier("d1full[%d]" % d, 2) for d in range(nd)]
        self.d1empty = [Barrier("d1empty[%d]" % d, 4) for d in range(nd)]
        # one A2-full barrier per (warpgroup, GEMM2 stream): each is waited for
        # by one stream, phase after phase
        self.a2full = [[Barrier("a2full[%d][%d]" % (b, v), 4) for v in range(2)] for b in range(nwg)]
        self.lcm = nwg if nwg % 2 == 0 else 2 * nwg
        self.a2empty = [Barrier("a2empty[%d]" % b) for b in range(nwg)]
        self.d2full = [[Barrier("d2full[%d][%d]" % (w, b)) for b in range(nb2)] for w in range(2)]
        self.d2empty = [[Barrier("d2empty[%d][%d]" % (w, b), 4) for b in range(nb2)] for w in range(2)]
        self.drain = [Barrier("drain[%d]" % u) for u in range(3)]
        self.drain2 = [Barrier("drain2[%d]" % w) for w in range(2)]
        # data
        self.stage = [None] * ns  # (tile, landed)
        self.dirs = [None] * 2  # (item, landed)
        self.d1 = [None] * nd  # tile whose projections the buffer holds
        self.d1_read = {}  # tile -> set of warps that loaded it
        self.a2 = [[None] * 4 for _ in range(nwg)]  # per buffer, per lane quarter: tile
        self.d2 = [[None] * nb2 for _ in range(2)]  # per stream, buffer: (period, set of tiles)
        self.mag_read = {}  # tile -> set of warps that read its magnitudes (from the stage)
        self.stage_seen = set()  # tiles whose landed stage a GEMM1 warp has seen
        self.folded = {}  # (stream, period) -> set of fold warps
        self.g1_done = set()
        self.g2_done = set()
        self.g1_of_item_done = {}
        # async work
        self.mma_q = {"g1": [], "g2_0": [], "g2_1": []}
        self.tma = []  # pending copies
        self.progs = {"tma": self._tma_warp(), "g1": self._gemm1_warp(),
                      "g2_0": self._gemm2_warp(0), "g2_1": self._gemm2_warp(1)}
        for wg in range(nwg):
            for q in range(4):
                self.progs[("r", wg, q)] = self._rounding_warp(wg, q)
        for q in range(4):
            self.progs[("f", q)] = self._fold_warp(q)
        self.finished = set()
        self.blocked = {}

    def _wait(self, who, bar, k, may_fail=True):
        bar.start_wait(who, k)
        return ("wait", bar, k, may_fail)

    # ------------------------------------------------------------ programs
    def _tma_warp(self):
        ns = self.ns
        lg = 0
        ok = True
        issued_dirs = 0
        for k in range(self.n_items):
            if k >= 2:
                ok = yield self._wait("tma", self.dempty[k % 2], (k - 2) // 2)
                if not ok:
                    break
            old = k - 2
            if old >= 0 and len(self.g1_of_item_done.get(old, ())) != self.items[old]:
                raise ProtocolError("direction buffer %d refilled with item %d before item %d's GEMM1s executed"
                                    % (k % 2, k, old))
            self.dfull[k % 2].expect_tx(1)
            self.dfull[k % 2].arrive()
            self.tma.append(("dirs", k % 2, k, self.dfull[k % 2]))
            issued_dirs += 1
            for j in range(self.items[k]):
                g = lg
                s = g % ns
                if g >= ns:
                    k_wait = g // ns - 1
                    if self.mut == "refill_early":
                        k_wait -= 1
                    if k_wait >= 0:
                        ok = yield self._wait("tma", self.sempty[s], k_wait)
                        if not ok:
                            break
                    old = g - ns
                    if len(self.mag_read.get(old, ())) != 4:
                        raise ProtocolError("stage %d refilled with tile %d before tile %d's magnitudes were read"
                                            % (s, g, old))
                    if not (old in self.g1_done and old in self.g2_done):
                        raise ProtocolError("stage %d refilled with tile %d before both GEMMs of tile %d executed"
                                            % (s, g, old))
                self.sfull[s].expect_tx(1)
                self.sfull[s].arrive()
                self.tma.append(("stage", s, g, self.sfull[s]))
                lg += 1
            if not ok:
                break
        if not ok:
            self.abort = True
        # drain: the copies still in flight land before the teardown
        for t in range(max(0, lg - ns), lg):
            yield self._wait("tma", self.sfull[t % ns], t // ns, may_fail=False)
        for t in range(max(0, issued_dirs - 2), issued_dirs):
            yield self._wait("tma", self.dfull[t % 2], t // 2, may_fail=False)

    def _gemm1_warp(self):
        who = "g1"
        q = self.mma_q[who]
        ns, nd = self.ns, self.nd
        g = 0
        ok = True
        for k in range(self.n_items):
            ok = yield self._wait(who, self.dfull[k % 2], k // 2)
            if not ok:
                break
            for j in range(self.items[k]):
                ok = yield self._wait(who, self.sfull[g % ns], g // ns)
                if ok and g >= nd and self.mut != "no_d1_wait":
                    ok = yield self._wait(who, self.d1empty[g % nd], g // nd - 1)
                if not ok:
                    break
                if self.stage[g % ns] != (g, True):
                    raise ProtocolError("%s saw stage %d holding %r for tile %d" % (who, g % ns, self.stage[g % ns], g))
                self.stage_seen.add(g)
                self.d1full[g % nd].arrive()
                q.append(("gemm1", g))
                q.append(("commit", self.d1full[g % nd]))
                g += 1
            if not ok:
                break
            q.append(("commit", self.dempty[k % 2]))
        if not ok:
            self.abort = True
        if self.mut != "no_drain":
            q.append(("commit", self.drain[2]))
            yield self._wait(who, self.drain[2], 0, may_fail=False)

    def _gemm2_warp(self, v):
        who = "g2_%d" % v
        q = self.mma_q[who]
        nb2 = self.nb2
        ok = True
        for g in range(v, self.T, 2):
            sv, p = self.period_of[g]
            if self.first[g] and p >= nb2 and self.mut != "no_d2_wait":
                ok = yield self._wait(who, self.d2empty[v][p % nb2], p // nb2 - 1)
                if not ok:
                    break
            w = g % self.nwg
            ok = yield self._wait(who, self.a2full[w][v], g // self.lcm)
            if not ok:
                break
            q.append(("gemm2", g))
            q.append(("commit", self.a2empty[w]))
            q.append(("commit", self.sempty[g % self.ns]))
            if self.last[g]:
                q.append(("commit", self.d2full[v][p % nb2]))
        if not ok:
            self.abort = True
        q.append(("commit", self.drain[v]))
        yield self._wait(who, self.drain[v], 0, may_fail=False)

    def _rounding_warp(self, wg, q):
        who = ("r", wg, q)
        nd = self.nd
        ok = True
        for g in range(wg, self.T, self.nwg):
            d = g % nd
            if self.mut == "release_early":
                self.d1empty[d].arrive()
            ok = yield self._wait(who, self.d1full[d], g // nd)
            if not ok:
                break
            st = self.stage[g % self.ns]
            if g not in self.stage_seen or st != (g, True):
                raise ProtocolError("%r reads magnitudes of tile %d from stage holding %r" % (who, g, st))
            if self.d1[d] != g:
                raise ProtocolError("%r reads D1[%d] holding tile %r, wants %d" % (who, d, self.d1[d], g))
            self.d1_read.setdefault(g, set()).add(who)
            if self.mut != "release_early":
                self.d1empty[d].arrive()
            yield ("step",)  # the rounding itself
            # the last chunk's magnitudes are read after the release
            st = self.stage[g % self.ns]
            if st != (g, True):
                raise ProtocolError("%r reads magnitudes of tile %d from stage holding %r" % (who, g, st))
            self.mag_read.setdefault(g, set()).add(who)
            prev = g - self.nwg
            if prev >= 0 and self.mut != "no_a2_wait":
                ok = yield self._wait(who, self.a2empty[wg], g // self.nwg - 1)
                if not ok:
                    break
            if prev >= 0 and prev not in self.g2_done:
                raise ProtocolError("%r overwrites A2[%d] before GEMM2(%d) read it" % (who, wg, prev))
            self.a2[wg][q] = g
            self.a2full[wg][g % 2].arrive()
        if not ok:
            self.abort = True

    def _fold_warp(self, q):
        who = ("f", q)
        ok = True
        for per_item in self.item_periods:
            for i in range(max(len(per_item[0]), len(per_item[1]))):
                for w in range(2):
                    if i >= len(per_item[w]):
                        continue
                    p = per_item[w][i]
                    nb2 = self.nb2
                    ok = yield self._wait(who, self.d2full[w][p % nb2], p // nb2)
                    if not ok:
                        break
                    cur = self.d2[w][p % nb2]
                    if cur is None or cur[0] != p or cur[1] != self.period_tiles[(w, p)]:
                        raise ProtocolError("%r folds period %d of stream %d from D2 holding %r" % (who, p, w, cur))
                    self.folded.setdefault((w, p), set()).add(who)
                    self.d2empty[w][p % nb2].arrive()
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            self.abort = True

    # ----------------------------------------------------------- async ops
    def _exec_gemm1(self, t):
        s = t % self.ns
        item = self.tiles[t][0]
        d = t % self.nd
        if self.stage[s] != (t, True):
            raise ProtocolError("GEMM1(%d) reads stage %d holding %r" % (t, s, self.stage[s]))
        if self.dirs[item % 2] != (item, True):
            raise ProtocolError("GEMM1(%d) reads directions %r, wants item %d" % (t, self.dirs[item % 2], item))
        old = t - self.nd
        if old >= 0 and len(self.d1_read.get(old, ())) != 4:
            raise ProtocolError("GEMM1(%d) overwrites D1[%d] before every warp read D1(%d)" % (t, d, old))
        self.d1[d] = t
        self.g1_done.add(t)
        self.g1_of_item_done.setdefault(item, set()).add(t)

    def _exec_gemm2(self, t):
        s = t % self.ns
        b = t % self.nwg
        if self.stage[s] != (t, True):
            raise ProtocolError("GEMM2(%d) reads stage %d holding %r" % (t, s, self.stage[s]))
        if self.a2[b] != [t] * 4:
            raise ProtocolError("GEMM2(%d) reads A2[%d] holding tiles %r" % (t, b, self.a2[b]))
        w, p = self.period_of[t]
        nb2 = self.nb2
        if self.first[t]:
            if p >= nb2 and len(self.folded.get((w, p - nb2), ())) != 4:
                raise ProtocolError("GEMM2(%d) starts period %d of stream %d before period %d was folded"
                                    % (t, p, w, p - nb2))
            self.d2[w][p % nb2] = (p, {t})
        else:
            cur = self.d2[w][p % nb2]
            if cur is None or cur[0] != p:
                raise ProtocolError("GEMM2(%d) accumulates into D2 of period %r" % (t, cur))
            cur[1].add(t)
        self.g2_done.add(t)

    # ----------------------------------------------------------- scheduler
    def _enabled(self):
        agents = []
        for w in self.progs:
            if w in self.finished:
                continue
            req = self.blocked.get(w)
            if req is None or req[0] == "step":
                agents.append(("warp", w, None))
            elif req[0] == "wait":
                bar, k, may_fail = req[1], req[2], req[3]
                if bar.ready(k):
                    agents.append(("warp", w, True))
                elif may_fail and self.abort:
                    agents.append(("warp", w, False))  # the abort flag: give up at once
                elif may_fail and self.fail_prob > 0 and self.rng.random() < self.fail_prob:
                    agents.append(("warp", w, False))  # the bounded wait runs out
        for q in self.mma_q:
            if self.mma_q[q]:
                agents.append(("mma", q, None))
        for idx in range(len(self.tma)):
            agents.append(("tma", idx, None))
        if self.slow_mma and self.mma_q["g1"]:
            agents.append(("tick", None, None))
        return agents

    def _step_warp(self, w, value):
        req = self.blocked.pop(w, None)
        if req is not None and req[0] == "wait":
            req[1].end_wait(w)
        try:
            nxt = self.progs[w].send(value) if req is not None else next(self.progs[w])
        except StopIteration:
            self.finished.add(w)
            return
        self.blocked[w] = nxt

    def _step_mma(self, q):
        op = self.mma_q[q].pop(0)
        if op[0] == "gemm1":
            self._exec_gemm1(op[1])
        elif op[0] == "gemm2":
            self._exec_gemm2(op[1])
        else:  # commit: every earlier operation of this warp has executed
            op[1].arrive()

    def _step_tma(self, idx):
        kind, slot, content, bar = self.tma.pop(idx)
        if kind == "stage":
            self.stage[slot] = (content, True)
        else:
            self.dirs[slot] = (content, True)
        bar.complete_tx(1)

    def run(self, max_steps=400000):
        for _ in range(max_steps):
            if len(self.finished) == len(self.progs):
                if self.tma or any(self.mma_q.values()):
                    raise ProtocolError("teardown with work in flight: %d copies, MMA queues %r"
                                        % (len(self.tma), {q: len(v) for q, v in self.mma_q.items()}))
                if not self.abort and len(self.g2_done) != self.T:
                    raise ProtocolError("finished with %d of %d tiles scored" % (len(self.g2_done), self.T))
                return
            agents = self._enabled()
            if not agents:
                raise ProtocolError("deadlock: warps %r blocked on %r" % (
                    sorted((str(w) for w in self.progs if w not in self.finished)),
                    {str(w): (r[1].name, r[2]) if r[0] == "wait" else r for w, r in self.blocked.items()}))
            weights = [1.0 if ag[0] == "warp" else
                       (0.002 if self.slow_mma and ag[:2] == ("mma", "g1") else self.async_weight)
                       for ag in agents]
            kind, a, value = self.rng.choices(agents, weights)[0]
            if kind == "tick":
                continue
            if kind == "warp":
                self._step_warp(a, value)
            elif kind == "mma":
                self._step_mma(a)
            else:
                self._step_tma(a)
        raise ProtocolError("no progress within %d steps" % max_steps)


def check(items, ns, nd, flush, seed, mutation=None, fail_prob=0.0, async_weight=1.0, slow_mma=False, nwg=None,
          nb2=1):
    """Run one random schedule of a CTA over `items`; raises ProtocolError.
    Returns the CTA (its `abort` flag says whether a wait gave up)."""
    cta = Cta(items, ns, nwg or nd, flush, seed, mutation, fail_prob, async_weight, slow_mma, nwg or nd, nb2)
    cta.run()
    return cta
