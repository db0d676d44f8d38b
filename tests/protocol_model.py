"""Executable model of the per-worker synchronisation protocol of score_tc_kernel.

Test infrastructure (plain Python, no GPU).  The model mirrors, step for step,
the program one worker of the tensor-core scoring kernel runs:

* four rounding warps; warp 0 also issues GEMM1, warp 2 GEMM2, and one lane
  of warp 1 (the loader) issues the TMA copies;
* the tcgen05 operations (MMAs and commits) of warps 0 and 2, which execute
  in issue order per issuing warp and in any order across the two warps; a
  commit arrives on its mbarrier once every earlier operation of its warp
  has executed;
* the TMA copies, which complete in any order;
* the mbarriers (arrival count, transaction bytes, completed phases) with
  their parity waits, and the warpgroup rendezvous.

A seeded random scheduler runs one enabled agent at a time (a warp, the head
of an MMA queue, a pending copy).  The checker raises ProtocolError on

* a deadlock: nothing can run and some warp has not finished;
* a parity wait that could alias: a warp waits for phase k of a barrier that
  has already completed phase k + 1 (mbarrier.try_wait.parity cannot tell
  phase k from phase k + 2, so such a wait would block or pass on the wrong
  phase);
* a data hazard: an operand read before the data it needs was written
  (D1 of the wrong tile, a stage or direction buffer not yet landed, A2 or D2
  holding the wrong tiles), or a buffer overwritten before its last reader
  has consumed it.

`fail_prob` > 0 also exercises the failure path: a wait that is not yet
satisfied may give up (a bounded wait running out), exactly as the kernel's
waits do, and then the warp carries `bad` to the rendezvous, which every warp
leaves together (bar.red.or), or sets the CTA's abort flag, which makes every
other unsatisfied wait give up at once.  The checker then also requires that
no MMA or copy is outstanding when the last warp reaches the teardown (TMEM is
freed and the CTA exits there).

`mutation` plants one known mistake in the protocol (the checker must catch
it): "refill_early" refills a stage one tile too soon, "no_a2_wait" stores A2
without waiting for the previous GEMM2, "gemm2_early" issues GEMM2 before the
rendezvous, "no_drain" lets warp 0 skip its drain.
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
        self.waiters[who] = k

    def ready(self, k):
        return self.done >= k + 1

    def end_wait(self, who):
        self.waiters.pop(who, None)


def make_items(rng, n_items, max_tiles):
    return [rng.randint(1, max_tiles) for _ in range(n_items)]


class Worker:
    """One worker of the kernel; `items` is the number of tiles of each item."""

    def __init__(self, items, nst, flush, seed, mutation=None, fail_prob=0.0, async_weight=1.0, slow_mma0=False):
        self.rng = random.Random(seed)
        self.async_weight = async_weight  # < 1: MMAs and copies lag behind the warps
        self.slow_mma0 = slow_mma0  # warp 0's MMAs far slower than everything else
        self.fail_prob = fail_prob
        self.abort = False
        self.nst = nst
        self.F = flush
        self.mut = mutation
        # the worker's tile sequence: (item, j, ntile)
        self.tiles = [(i, j, nt) for i, nt in enumerate(items) for j in range(nt)]
        self.T = len(self.tiles)
        self.n_items = len(items)
        # barriers
        self.full = [Barrier("full[%d]" % s) for s in range(nst)]
        self.a1_full = [Barrier("a1_full[%d]" % b) for b in range(2)]
        self.d1_full = Barrier("d1_full")
        self.d2_ready = Barrier("d2_ready")
        self.a2_free = Barrier("a2_free")
        self.drain = Barrier("drain")
        self.drain2 = Barrier("drain2")
        # named barrier (rendezvous) state
        self.bar_gen = 0
        self.bar_count = 0
        self.bar_or = False
        self.bar_result = {}  # generation -> OR of the warps' flags
        # data
        self.stage = [None] * nst  # (tile, landed)
        self.dirs = [None] * 2  # (item, landed)
        self.d1 = None
        self.d1_read = {}  # tile -> set of warps
        self.a2 = [None] * 4  # tile per lane quarter
        self.d2 = None  # (period, set of tiles)
        self.folded = {}  # period -> set of warps
        self.g1_done = set()
        self.g2_done = set()
        self.g1_of_item_done = {}  # item -> tiles whose GEMM1 executed
        # async work
        self.mma_q = {0: [], 2: []}
        self.tma = []  # pending copies
        # periods: tile -> period index, period -> tiles
        self.period_of = {}
        self.period_tiles = {}
        pos, p = 0, 0
        for g, (i, j, nt) in enumerate(self.tiles):
            self.period_of[g] = p
            self.period_tiles.setdefault(p, set()).add(g)
            last = pos == flush - 1 or j == nt - 1
            if last:
                p += 1
                pos = 0
            else:
                pos += 1
        self.finished = set()
        self.gens = {w: self._rounding_warp(w) for w in range(4)}
        self.blocked = {}  # warp -> predicate that must hold to resume

    # ---------------------------------------------------------------- helpers
    def _flags(self, g, pos):
        i, j, nt = self.tiles[g]
        first = pos == 0
        item_end = j == nt - 1
        last = pos == self.F - 1 or item_end
        has_next = g + 1 < self.T
        return first, item_end, last, has_next

    def _wait(self, who, bar, k, may_fail=True):
        bar.start_wait(who, k)
        return ("wait", bar, k, may_fail)

    # ------------------------------------------------------------- data paths
    def _tma_stage(self, t):
        s = t % self.nst
        old = t - self.nst
        if old >= 0 and not (old in self.g1_done and old in self.g2_done):
            raise ProtocolError("stage %d refilled with tile %d before both GEMMs of tile %d executed" % (s, t, old))
        bar = self.full[s]
        bar.expect_tx(1)
        bar.arrive()
        self.tma.append(("stage", s, t, bar))

    def _tma_dirs(self, item):
        b = item % 2
        old = item - 2
        if old >= 0:
            n_old = sum(1 for (i, _, _) in self.tiles if i == old)
            if len(self.g1_of_item_done.get(old, ())) != n_old:
                raise ProtocolError("direction buffer %d refilled with item %d before item %d's GEMM1s executed"
                                    % (b, item, old))
        bar = self.a1_full[b]
        bar.expect_tx(1)
        bar.arrive()
        self.tma.append(("dirs", b, item, bar))

    def _exec_gemm1(self, t):
        s = t % self.nst
        item = self.tiles[t][0]
        if self.stage[s] != (t, True):
            raise ProtocolError("GEMM1(%d) reads stage %d holding %r" % (t, s, self.stage[s]))
        if self.dirs[item % 2] != (item, True):
            raise ProtocolError("GEMM1(%d) reads directions %r, wants item %d" % (t, self.dirs[item % 2], item))
        if t > 0 and len(self.d1_read.get(t - 1, ())) != 4:
            raise ProtocolError("GEMM1(%d) overwrites D1 before every warp read D1(%d)" % (t, t - 1))
        self.d1 = t
        self.g1_done.add(t)
        self.g1_of_item_done.setdefault(item, set()).add(t)

    def _exec_gemm2(self, t, first):
        s = t % self.nst
        if self.stage[s] != (t, True):
            raise ProtocolError("GEMM2(%d) reads stage %d holding %r" % (t, s, self.stage[s]))
        if self.a2 != [t] * 4:
            raise ProtocolError("GEMM2(%d) reads A2 holding tiles %r" % (t, self.a2))
        p = self.period_of[t]
        if first:
            if p > 0 and len(self.folded.get(p - 1, ())) != 4:
                raise ProtocolError("GEMM2(%d) starts period %d before period %d was folded" % (t, p, p - 1))
            self.d2 = (p, {t})
        else:
            if self.d2 is None or self.d2[0] != p:
                raise ProtocolError("GEMM2(%d) accumulates into D2 of period %r" % (t, self.d2))
            self.d2[1].add(t)
        self.g2_done.add(t)

    # ------------------------------------------------------------ warp program
    def _rounding_warp(self, w):
        # Every wait is `ok = yield ("wait", bar, k)`: True once the phase has
        # completed, False when it gives up (timeout or abort flag).
        nst = self.nst
        T = self.T
        lg = la = cg = ca = 0
        if w == 1 and T > 0:  # loader prologue
            for item in range(min(2, self.n_items)):
                self._tma_dirs(item)
                la += 1
            while lg < nst and lg < T:
                self._tma_stage(lg)
                lg += 1
        if w == 0 and T > 0:  # GEMM1(0) once its operands have landed
            ok = yield self._wait(w, self.a1_full[0], 0)
            ca += 1
            if ok:
                ok = yield self._wait(w, self.full[0], 0)
                cg += 1
            if ok:
                self.mma_q[0].append(("gemm1", 0))
                self.mma_q[0].append(("commit", self.d1_full))
            else:
                self.abort = True
        pos = 0
        pe = 0
        bad = False
        for g in range(T):
            first, item_end, last, has_next = self._flags(g, pos)
            if not bad:
                bad = not (yield self._wait(w, self.d1_full, g))
            if not bad:
                if self.d1 != g:
                    raise ProtocolError("warp %d reads D1 holding tile %r, wants %d" % (w, self.d1, g))
                self.d1_read.setdefault(g, set()).add(w)
                if g > 0 and self.mut != "no_a2_wait":
                    bad = not (yield self._wait(w, self.a2_free, g - 1))
                if not bad:
                    if g > 0 and (g - 1) not in self.g2_done:
                        raise ProtocolError("warp %d overwrites A2 before GEMM2(%d) read it" % (w, g - 1))
                    self.a2[w] = g
                    if w == 2 and self.mut == "gemm2_early":
                        self._issue_gemm2(g, first, last)
            if (yield ("rendezvous", bad)):
                break  # every warp leaves here together
            if w == 1:
                limit = g + nst if self.mut == "refill_early" else g - 1 + nst
                while lg <= limit and lg < T:
                    self._tma_stage(lg)
                    lg += 1
                if item_end and la < self.n_items:
                    self._tma_dirs(la)
                    la += 1
            if w == 0 and has_next:
                ok = True
                if item_end:
                    ok = yield self._wait(w, self.a1_full[ca % 2], ca // 2)
                    ca += 1
                if ok:
                    ok = yield self._wait(w, self.full[cg % nst], cg // nst)
                    cg += 1
                if ok:
                    self.mma_q[0].append(("gemm1", g + 1))
                    self.mma_q[0].append(("commit", self.d1_full))
                else:
                    self.abort = True
            if w == 2 and self.mut != "gemm2_early":
                self._issue_gemm2(g, first, last)
            if last:
                bad = not (yield self._wait(w, self.d2_ready, pe))
                if not bad:
                    p = self.period_of[g]
                    if self.d2 is None or self.d2[0] != p or self.d2[1] != self.period_tiles[p]:
                        raise ProtocolError("warp %d folds period %d from D2 holding %r" % (w, p, self.d2))
                    self.folded.setdefault(p, set()).add(w)
                pe += 1
            pos = 0 if last else pos + 1
        if bad:
            self.abort = True
        # drain: the MMAs of warps 0 and 2 and the loader's copies complete
        # before TMEM is freed (these waits never give up early)
        if w == 0 and self.mut != "no_drain":
            self.mma_q[0].append(("commit", self.drain))
            yield self._wait(w, self.drain, 0, may_fail=False)
        if w == 2:
            self.mma_q[2].append(("commit", self.drain2))
            yield self._wait(w, self.drain2, 0, may_fail=False)
        if w == 1:
            for t in range(max(0, lg - nst), lg):
                yield self._wait(w, self.full[t % nst], t // nst, may_fail=False)
            for t in range(max(0, la - 2), la):
                yield self._wait(w, self.a1_full[t % 2], t // 2, may_fail=False)

    def _issue_gemm2(self, g, first, last):
        self.mma_q[2].append(("gemm2", g, first))
        if last:
            self.mma_q[2].append(("commit", self.d2_ready))
        self.mma_q[2].append(("commit", self.a2_free))

    # --------------------------------------------------------------- scheduler
    def _enabled(self):
        agents = []
        for w in range(4):
            if w in self.finished:
                continue
            req = self.blocked.get(w)
            if req is None:
                agents.append(("warp", w, None))
            elif req[0] == "wait":
                bar, k, may_fail = req[1], req[2], req[3]
                if bar.ready(k):
                    agents.append(("warp", w, True))
                elif may_fail and self.abort:
                    agents.append(("warp", w, False))  # the abort flag: give up at once
                elif may_fail and self.fail_prob > 0 and self.rng.random() < self.fail_prob:
                    agents.append(("warp", w, False))  # the bounded wait runs out
            elif req[0] == "rendezvous" and req[1] in self.bar_result:
                agents.append(("warp", w, self.bar_result[req[1]]))
        for q in (0, 2):
            if self.mma_q[q]:
                agents.append(("mma", q, None))
        for idx in range(len(self.tma)):
            agents.append(("tma", idx, None))
        if self.slow_mma0 and self.mma_q[0]:
            agents.append(("tick", None, None))  # time passes, nothing completes
        return agents

    def _step_warp(self, w, value):
        req = self.blocked.pop(w, None)
        if req is not None and req[0] == "wait":
            req[1].end_wait(w)
        try:
            nxt = self.gens[w].send(value) if req is not None else next(self.gens[w])
        except StopIteration:
            self.finished.add(w)
            return
        if nxt[0] == "rendezvous":
            gen = self.bar_gen
            self.bar_or = self.bar_or or bool(nxt[1])
            self.bar_count += 1
            if self.bar_count == 4:
                self.bar_result[gen] = self.bar_or
                self.bar_count = 0
                self.bar_or = False
                self.bar_gen += 1
            self.blocked[w] = ("rendezvous", gen)
        else:
            self.blocked[w] = nxt

    def _step_mma(self, q):
        op = self.mma_q[q].pop(0)
        if op[0] == "gemm1":
            self._exec_gemm1(op[1])
        elif op[0] == "gemm2":
            self._exec_gemm2(op[1], op[2])
        else:  # commit: every earlier operation of this warp has executed
            op[1].arrive()

    def _step_tma(self, idx):
        kind, slot, content, bar = self.tma.pop(idx)
        if kind == "stage":
            self.stage[slot] = (content, True)
        else:
            self.dirs[slot] = (content, True)
        bar.complete_tx(1)

    def run(self, max_steps=200000):
        for _ in range(max_steps):
            if len(self.finished) == 4:
                # the teardown: TMEM is freed and the CTA exits
                if self.tma or self.mma_q[0] or self.mma_q[2]:
                    raise ProtocolError("teardown with work in flight: %d copies, MMA queues %r"
                                        % (len(self.tma), {q: len(v) for q, v in self.mma_q.items()}))
                return
            agents = self._enabled()
            if not agents:
                raise ProtocolError("deadlock: warps %r blocked on %r" % (
                    sorted(set(range(4)) - self.finished),
                    {w: (r[1].name, r[2]) if r[0] == "wait" else r for w, r in self.blocked.items()}))
            weights = [1.0 if ag[0] == "warp" else
                       (0.002 if self.slow_mma0 and ag[:2] == ("mma", 0) else self.async_weight) for ag in agents]
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


def check(items, nst, flush, seed, mutation=None, fail_prob=0.0, async_weight=1.0, slow_mma0=False):
    """Run one random schedule of a worker over `items`; raises ProtocolError.
    Returns the worker (its `abort` flag says whether a wait gave up)."""
    wk = Worker(items, nst, flush, seed, mutation, fail_prob, async_weight, slow_mma0)
    wk.run()
    return wk
