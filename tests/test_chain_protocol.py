"""The wait and exit protocol of the coarse chain kernels, emulated on the CPU.

k_coarse_solve and k_seg_chain share one protocol (coarse.cu: chain_init, ring_produce,
ring_wait, chain_exit): per CTA a producer lane fills a ring of S shared-memory slots with bulk
copies (mbarrier "full", one arrival plus the bytes), consumer warps release each slot on
"empty" (one arrival per warp) after its copy has landed, and every step's row values are pushed
into every CTA of the cluster with st.async, completing bytes on the receiver's barrier rx[s]
(one barrier per step, armed once for B values when the kernel starts). Every wait is bounded;
a wait that runs out flags the CTA's error word.

The emulation restates that control flow step by step (generators stand for the producer lane
and the consumer warps; one poll per tick) against a model of the mbarrier (phase, pending
arrivals, transaction bytes) and runs it with faults injected on the host side of the model:
a bulk copy or a peer's store that lands late (after one wait bound has run out), a consumer
warp that stalls, a copy that never lands. It checks what the kernels rely on:
  * no CTA exits while an asynchronous copy or store into its shared memory is in flight
    (except one that lands later than the exit waits' bound after the exit barrier, such as a
    copy that never lands at all, which nothing could wait for; the faults here delay by up to
    two wait bounds, inside the exit waits' four);
  * once a timeout is flagged, the producer issues no further copy;
  * a slot never holds two copies in flight (so the parity waits stay unambiguous);
  * no barrier ever receives an arrival beyond its expected count;
  * the run ends within a bounded number of ticks, with the error flagged exactly when a
    fault made a wait run out.
"""
import pytest

KW = 400            # wait bound on the normal path (kWaitPolls, scaled down)
KW_ERR = 20         # in-loop receive waits after an error (kWaitPollsAfterError)
KDRAIN = 4 * KW     # chain_exit's waits (kDrainPolls)
COPY_LAT, PUSH_LAT = 6, 4


class MBar:
    """mbarrier: a phase completes when its pending arrivals and transaction bytes reach zero."""

    def __init__(self, count):
        self.count, self.pending, self.tx, self.phase = count, count, 0, 0

    def _complete(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def arrive(self):
        assert self.pending > 0, "arrival on a phase with no pending arrivals"
        self.pending -= 1
        self._complete()

    def expect_tx(self, nbytes):           # mbarrier.arrive.expect_tx
        self.tx += nbytes
        self.arrive()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        self._complete()

    def done(self, parity):                # try_wait.parity: the phase of that parity completed
        return (self.phase & 1) != parity


class Sim:
    def __init__(self, CS=3, nwc=2, S=2, nchunk=2, nsteps=6, tm=1, B=7, faults=(), skip_after_error=False):
        self.skip_after_error = skip_after_error   # the earlier protocol: waits skipped once flagged
        self.CS, self.nwc, self.S, self.nchunk, self.nsteps, self.tm, self.B = CS, nwc, S, nchunk, nsteps, tm, B
        self.U = max(0, nsteps - tm) * nchunk
        self.faults = dict(faults)
        self.t = 0
        self.events = []
        self.ctas = [self._cta(r) for r in range(CS)]
        self.cluster = {"arrived": 0, "gen": 0}
        self.nthreads = CS * (nwc + 1)

    def _cta(self, rank):
        R = (self.B + self.CS - 1) // self.CS
        nr = max(0, min(self.B, rank * R + R) - rank * R)
        return {"rank": rank, "nr": nr, "full": [MBar(1) for _ in range(self.S)],
                "empty": [MBar(self.nwc) for _ in range(self.S)], "rx": self._rx(),
                "s_err": 0, "s_issued": self.U, "inflight": set(), "slot_busy": [None] * self.S,
                "issued_after_err": 0, "exited": 0, "lost": set()}

    def _rx(self):                          # chain_init: one armed receive barrier per gathering step
        bars = [MBar(1) for _ in range(max(0, self.nsteps - 1))]
        for b in bars:
            b.expect_tx(8 * self.B)
        return bars

    # ---- asynchronous operations (land after a latency; a fault may delay or drop them)
    def _after(self, delay, fn):
        self.events.append((self.t + delay, fn))

    def issue_copy(self, cta, slot, u):
        assert cta["slot_busy"][slot] is None, "two copies in flight into one slot"
        if cta["s_err"]:
            cta["issued_after_err"] += 1
        nbytes = 8 * cta["nr"] * 4
        cta["full"][slot].expect_tx(nbytes)
        op = ("copy", cta["rank"], u)
        cta["slot_busy"][slot] = op
        fault = self.faults.get(op)
        if fault == "lost":
            cta["lost"].add(op)
            return
        cta["inflight"].add(op)

        def land():
            cta["inflight"].discard(op)
            cta["slot_busy"][slot] = None
            cta["full"][slot].complete_tx(nbytes)
        self._after(COPY_LAT + (fault or 0), land)

    def push(self, src, w, s):
        rows = len(range(w, src["nr"], self.nwc))
        if rows == 0:
            return                             # a warp with no rows of the slice stores nothing
        for dst in self.ctas:
            op = ("push", src["rank"], w, s, dst["rank"])
            dst["inflight"].add(op)

            def land(dst=dst, op=op):
                assert not dst["exited"], "a store landed in a CTA that had exited"
                dst["inflight"].discard(op)
                dst["rx"][s].complete_tx(8 * rows)
            self._after(PUSH_LAT + self.faults.get(("push", src["rank"], w, s), 0), land)

    # ---- the kernels' waits
    def wait(self, cta, bar, parity, polls=KW):   # (chain_exit passes KDRAIN)
        if bar.done(parity):
            return True
        if self.skip_after_error and cta["s_err"]:
            return False
        for _ in range(polls):
            yield
            if bar.done(parity):
                return True
        cta["s_err"] = 1
        return False

    def ring_wait(self, cta, slot, parity, u):
        if u >= cta["s_issued"]:
            return False
        if self.skip_after_error and cta["s_err"]:
            return True
        if cta["full"][slot].done(parity):
            return True
        for i in range(KW):
            yield
            if cta["full"][slot].done(parity):
                return True
            if i % 64 == 63 and u >= cta["s_issued"]:
                return False
        cta["s_err"] = 1
        return False

    def cluster_sync(self):
        gen = self.cluster["gen"]
        self.cluster["arrived"] += 1
        if self.cluster["arrived"] == self.nthreads:
            self.cluster["arrived"] = 0
            self.cluster["gen"] += 1
        while self.cluster["gen"] == gen:
            yield

    # ---- ring_produce (lane 0 of the producer warp)
    def producer(self, cta):
        S, U = self.S, self.U
        issued = 0
        for u in range(U):
            slot = u % S
            if u >= S and not (yield from self.wait(cta, cta["empty"][slot], ((u // S) - 1) & 1)):
                break
            if cta["s_err"]:
                break
            self.issue_copy(cta, slot, u)
            issued = u + 1
        if issued < U:
            cta["s_issued"] = issued
        yield from self.chain_exit(cta, 0)

    # ---- consumer warp w (warp 0 holds thread 0, which arms the receive phases)
    def consumer(self, cta, w):
        stall = self.faults.get(("stall", cta["rank"], w))
        if stall:
            for _ in range(stall):
                yield
        S = self.S
        u = 0
        for s in range(self.nsteps):
            more = s + 1 < self.nsteps
            if s >= self.tm:
                for _ in range(self.nchunk):
                    slot = u % S
                    ok = yield from self.ring_wait(cta, slot, (u // S) & 1, u)
                    if ok:
                        cta["empty"][slot].arrive()            # released only after a landed copy
                    u += 1
            if more:
                self.push(cta, w, s)
                yield from self.wait(cta, cta["rx"][s], 0, KW_ERR if cta["s_err"] else KW)
        yield from self.chain_exit(cta, w + 1)

    def chain_exit(self, cta, thread):
        """After the cluster barrier, on the error path only, every thread of the CTA waits for
        its share (thread i: items i, i + nthreads, ...) of the receive barriers and of the
        ring slots' last issued copies."""
        yield from self.cluster_sync()
        if cta["s_err"]:
            nth = self.nwc + 1
            for s in range(thread, len(cta["rx"]), nth):
                yield from self.wait(cta, cta["rx"][s], 0, KDRAIN)
            issued = cta["s_issued"]
            for slot in range(thread, min(self.S, issued), nth):
                ul = slot + ((issued - 1 - slot) // self.S) * self.S
                yield from self.wait(cta, cta["full"][slot], (ul // self.S) & 1, KDRAIN)
        cta["exited_threads"] = cta.get("exited_threads", 0) + 1
        if cta["exited_threads"] == self.nwc + 1:
            assert cta["inflight"] == set(), ("exit with async writes in flight", cta["inflight"])
            cta["exited"] = 1

    def run(self, limit=200000):
        threads = []
        for cta in self.ctas:
            threads.append(self.producer(cta))
            threads += [self.consumer(cta, w) for w in range(self.nwc)]
        while threads:
            assert self.t < limit, "the protocol did not end"
            due = [e for e in self.events if e[0] <= self.t]
            self.events = [e for e in self.events if e[0] > self.t]
            for _, fn in due:
                fn()
            alive = []
            for th in threads:
                try:
                    next(th)
                    alive.append(th)
                except StopIteration:
                    pass
            threads = alive
            self.t += 1
        for _, fn in sorted(self.events, key=lambda e: e[0]):
            fn()                                               # anything still pending lands
        return self


GEOMS = [dict(CS=3, nwc=2, S=2, nchunk=2, nsteps=6, tm=1),      # phase A / k_coarse_solve forward
         dict(CS=2, nwc=3, S=3, nchunk=1, nsteps=5, tm=0),      # phase B / backward launch
         dict(CS=4, nwc=2, S=4, nchunk=3, nsteps=4, tm=1, B=13)]


@pytest.mark.parametrize("geom", GEOMS, ids=["segA", "segB", "wide"])
def test_protocol_without_faults_flags_nothing(geom):
    sim = Sim(**geom).run()
    for cta in sim.ctas:
        assert cta["s_err"] == 0 and cta["exited"] and cta["s_issued"] == sim.U
        assert all(b.tx == 0 for b in cta["full"] + cta["rx"]) and all(b.phase == 1 for b in cta["rx"])


LATE = KW + KW // 2         # lands after one wait bound has run out, before the drain's bound


@pytest.mark.parametrize("geom", GEOMS, ids=["segA", "segB", "wide"])
@pytest.mark.parametrize("fault", ["late_copy_first", "late_copy_mid", "late_push", "stalled_warp"])
def test_timeout_drains_before_exit(geom, fault):
    U = max(0, geom["nsteps"] - geom["tm"]) * geom["nchunk"]
    faults = {"late_copy_first": {("copy", 1, 0): LATE},
              "late_copy_mid": {("copy", 0, U // 2): LATE},
              "late_push": {("push", 1, 0, 1): LATE},
              "stalled_warp": {("stall", 0, 1): LATE}}[fault]
    sim = Sim(faults=faults, **geom).run()
    assert any(c["s_err"] for c in sim.ctas)                   # the fault made a wait run out
    for cta in sim.ctas:
        assert cta["exited"]                                   # (chain_exit checked: nothing in flight)
        assert cta["issued_after_err"] <= 0 or cta["s_issued"] < sim.U
        assert all(b is None for b in cta["slot_busy"])        # every issued copy was waited on


def test_no_copy_issued_after_a_flagged_timeout():
    """After the first flagged timeout in a CTA its producer issues nothing further."""
    sim = Sim(faults={("copy", 0, 1): LATE}, CS=2, nwc=2, S=2, nchunk=2, nsteps=8, tm=1)
    sim.run()
    assert sim.ctas[0]["s_err"] and sim.ctas[0]["issued_after_err"] == 0
    assert sim.ctas[0]["s_issued"] < sim.U


def test_lost_copy_ends_in_bounded_time():
    """A copy that never lands: every wait for it runs out, nothing else stays in flight,
    and the launch ends."""
    sim = Sim(faults={("copy", 2, 3): "lost"}, **GEOMS[0]).run()
    assert sim.ctas[2]["s_err"] and sim.ctas[2]["lost"]
    for cta in sim.ctas:
        assert cta["exited"]


@pytest.mark.parametrize("seed", range(12))
def test_random_late_operations(seed):
    """Late copies and stores at seeded random places (one to three per run)."""
    import random
    rnd = random.Random(seed)
    geom = GEOMS[seed % len(GEOMS)]
    sim0 = Sim(**geom)
    faults = {}
    for _ in range(rnd.randint(1, 3)):
        kind = rnd.choice(["copy", "push", "stall"])
        if kind == "copy" and sim0.U:
            faults[("copy", rnd.randrange(geom["CS"]), rnd.randrange(sim0.U))] = rnd.randint(KW + 1, 2 * KW - 50)
        elif kind == "push":
            faults[("push", rnd.randrange(geom["CS"]), rnd.randrange(geom["nwc"]),
                    rnd.randrange(geom["nsteps"] - 1))] = rnd.randint(KW + 1, 2 * KW - 50)
        else:
            faults[("stall", rnd.randrange(geom["CS"]), rnd.randrange(geom["nwc"]))] = rnd.randint(KW + 1, 2 * KW)
    sim = Sim(faults=faults, **geom).run()
    for cta in sim.ctas:
        assert cta["exited"] and all(b is None for b in cta["slot_busy"])


def test_skipping_waits_after_an_error_is_caught():
    """Negative control: the earlier protocol, in which every wait returned at once after the
    first timeout, lets a CTA exit with a copy still in flight; the emulation must see it."""
    with pytest.raises(AssertionError, match="in flight|exited|two copies"):
        Sim(faults={("copy", 0, 2): LATE}, skip_after_error=True, **GEOMS[1]).run()
