"""Serving loop: continuous batching over many streams with admission.

CPU tests drive the scheduler against a fake library that records what it is
asked to do.  The GPU tests replay a small trace through the CUDA library and
check that every stream's hits equal the oracle's for that stream's packets
concatenated, and equal the result of running the stream alone."""
import numpy as np
import pytest

from paper_1712_03560_gb300 import serve
from paper_1712_03560_gb300 import workloads as W


class FakeLib:
    """Stands in for the binding: slots, per-stream byte logs, no matching."""
    OASM_EBUSY, OASM_ENOMEM = -3, -2

    class OasmError(RuntimeError):
        def __init__(self, code):
            super().__init__(code)
            self.code = code

    def __init__(self, slots):
        self.slots = slots
        self.open = {}
        self.log = []          # (event, ...) in call order
        self.data = {}         # sid -> bytes fed in order (for the current occupant)
        self.ended = set()
        self.next_id = 0

    def oasm_create(self, patterns, ks, rules, cfg):
        return "ctx"

    def oasm_destroy(self, ctx):
        pass

    def oasm_open_stream(self, ctx):
        free = [s for s in range(self.slots) if s not in self.open]
        if not free:
            raise self.OasmError(self.OASM_EBUSY)
        s = free[0]
        self.open[s] = self.next_id
        self.next_id += 1
        self.data[s] = bytearray()
        self.log.append(("open", s))
        return s

    def oasm_open_streams(self, ctx, n):
        out = []
        for _ in range(n):
            try:
                out.append(self.oasm_open_stream(ctx))
            except self.OasmError:
                break
        return np.asarray(out, dtype=np.uint32)

    def oasm_end_streams(self, ctx, sids):
        for s in sids:
            self.oasm_end_stream(ctx, int(s))

    def oasm_close_streams(self, ctx, sids):
        for s in sids:
            self.oasm_close_stream(ctx, int(s))

    def oasm_close_stream(self, ctx, s):
        assert s in self.ended, "closed before its end was processed"
        self.log.append(("close", s, bytes(self.data[s])))
        del self.open[s]
        self.ended.discard(s)

    def oasm_feed_many(self, ctx, sids, buf, offs, lens):
        for s, o, n in zip(sids.tolist(), offs.tolist(), lens.tolist()):
            assert s in self.open and s not in self.ended
            self.data[s] += bytes(buf[o:o + n])
        self.log.append(("feed", len(sids)))

    def oasm_end_stream(self, ctx, s):
        self.ended.add(s)

    def oasm_step(self, ctx):
        self.log.append(("step",))

    def oasm_drain(self, ctx):
        from paper_1712_03560_gb300.binding import HIT_DTYPE
        return np.zeros(0, dtype=HIT_DTYPE)


@pytest.mark.parametrize("slots,budget", [(3, 1 << 30), (5, 3000), (64, 1 << 30), (2, 1500)])
def test_scheduler_feeds_every_packet_once_in_stream_order(slots, budget):
    tr = W.served(seed=3, n_streams=12, n_sig=4, gbps=1.0, duration=0.004, life=0.4)
    lib = FakeLib(slots)
    srv = serve.Server([b"AB"], [0], max_streams=slots, lib=lib, max_batch_bytes=budget)
    res = srv.replay(tr, realtime=False)
    texts = tr.stream_texts()
    closed = [e for e in lib.log if e[0] == "close"]
    # every stream that has packets was opened, got exactly its bytes in order, and closed
    got = sorted(e[2] for e in closed)
    want = sorted(bytes(t) for t in texts if t.size)
    assert got == want
    assert res["packets"] == tr.n_packets and res["fed_bytes"] == int(tr.lens.sum())
    assert res["p50_ms"] is not None and res["p99_ms"] >= res["p50_ms"]
    assert res["streams_admitted"] == sum(1 for t in texts if t.size)
    # never more open streams than slots
    live, peak = 0, 0
    for e in lib.log:
        live += {"open": 1, "close": -1}.get(e[0], 0)
        peak = max(peak, live)
    assert peak <= slots
    if slots < 12:
        assert res["max_waiting_streams"] > 0


class MemLimitedLib(FakeLib):
    """Admission refused by memory (OASM_ENOMEM) below the slot count."""

    def __init__(self, slots, mem_streams):
        super().__init__(slots)
        self.mem_streams = mem_streams

    def oasm_open_stream(self, ctx):
        if len(self.open) >= self.mem_streams:
            raise self.OasmError(self.OASM_ENOMEM)
        return super().oasm_open_stream(ctx)


def test_scheduler_waits_out_admission_refused_by_memory():
    """Host fault injection: the library refuses new streams for memory while
    slots are free; the scheduler keeps them waiting and still feeds every
    packet exactly once, in order."""
    tr = W.served(seed=5, n_streams=10, n_sig=4, gbps=1.0, duration=0.004, life=0.4)
    lib = MemLimitedLib(slots=8, mem_streams=3)
    srv = serve.Server([b"AB"], [0], max_streams=8, lib=lib, max_batch_bytes=4000)
    res = srv.replay(tr, realtime=False)
    got = sorted(e[2] for e in lib.log if e[0] == "close")
    assert got == sorted(bytes(t) for t in tr.stream_texts() if t.size)
    assert res["max_waiting_streams"] > 0
    live, peak = 0, 0
    for e in lib.log:
        live += {"open": 1, "close": -1}.get(e[0], 0)
        peak = max(peak, live)
    assert peak <= 3


class FailingStepLib(FakeLib):
    """A step that reports a device-wait timeout (OASM_ETIMEOUT) on its third call."""
    OASM_ETIMEOUT = -5

    def __init__(self, slots):
        super().__init__(slots)
        self.steps = 0

    def oasm_step(self, ctx):
        self.steps += 1
        if self.steps == 3:
            raise self.OasmError(self.OASM_ETIMEOUT)
        super().oasm_step(ctx)


def test_scheduler_surfaces_a_failed_step():
    """Host fault injection: a step that fails (a bounded device wait ran
    out) ends the replay with that error at once instead of hanging or
    dropping it."""
    tr = W.served(seed=6, n_streams=6, n_sig=4, gbps=1.0, duration=0.004, life=0.4)
    lib = FailingStepLib(6)
    srv = serve.Server([b"AB"], [0], max_streams=6, lib=lib, max_batch_bytes=2000)
    with pytest.raises(FakeLib.OasmError) as ei:
        srv.replay(tr, realtime=False)
    assert ei.value.code == FailingStepLib.OASM_ETIMEOUT
    assert lib.steps == 3


def test_scheduler_realtime_pacing_batches_arrivals():
    tr = W.served(seed=4, n_streams=8, n_sig=4, gbps=0.05, duration=0.05)
    lib = FakeLib(8)
    srv = serve.Server([b"AB"], [0], max_streams=8, lib=lib)
    res = srv.replay(tr, realtime=True)
    assert res["wall_s"] >= tr.times[-1] * 0.9
    assert res["steps"] >= 2
    assert np.isfinite(res["p99_ms"])


class NativeFake:
    """A fake library for the native serving loop (oasm_replay_ops): the same
    bookkeeping as FakeLib, called from C through the entry-point table.
    mem_streams < slots refuses admission for memory below the slot count;
    fail_step = n makes the n-th step report a device-wait timeout."""
    OASM_ETIMEOUT = -5

    def __init__(self, slots, mem_streams=None, fail_step=None):
        self.slots = slots
        self.mem = slots if mem_streams is None else mem_streams
        self.fail_step = fail_step
        self.open, self.data, self.ended, self.log = set(), {}, set(), []
        self.steps = 0
        self.pending = False

    def ops(self):
        import ctypes

        def open_streams(n, sids, n_opened):
            got = 0
            for s in range(self.slots):
                if got == n or len(self.open) >= self.mem:
                    break
                if s not in self.open:
                    self.open.add(s)
                    self.data[s] = bytearray()
                    self.log.append(("open", s))
                    sids[got] = s
                    got += 1
            n_opened[0] = got
            return 0

        def feed_many(n, sid, buf, off, ln):
            base = ctypes.addressof(buf.contents)
            for j in range(n):
                s = sid[j]
                assert s in self.open and s not in self.ended
                self.data[s] += ctypes.string_at(base + off[j], ln[j])
            self.pending = True
            return 0

        def end_streams(n, sids):
            for j in range(n):
                self.ended.add(sids[j])
            return 0

        def close_streams(n, sids):
            for j in range(n):
                s = sids[j]
                assert s in self.ended, "closed before its end was processed"
                self.log.append(("close", s, bytes(self.data[s])))
                self.open.discard(s)
                self.ended.discard(s)
            return 0

        def step_begin():
            self.steps += 1
            self.log.append(("step",))
            return 0

        def step_end():
            return self.OASM_ETIMEOUT if self.steps == self.fail_step else 0

        def ready(sid, n):
            n[0] = 0
            return 0

        def drain(out, cap, n):
            n[0] = 0
            return 0

        return dict(open_streams=open_streams, feed_many=feed_many, end_streams=end_streams,
                    close_streams=close_streams, step_begin=step_begin, step_end=step_end,
                    ready=ready, drain=drain)


def native_replay(tr, fake, budget):
    from paper_1712_03560_gb300 import binding as B
    return B.oasm_replay_ops(fake.ops(), tr.times, tr.streams, tr.offs, tr.lens, tr.last,
                             tr.payload, tr.n_streams, realtime=False, max_batch_bytes=budget)


def peak_open(log):
    live, peak = 0, 0
    for e in log:
        live += {"open": 1, "close": -1}.get(e[0], 0)
        peak = max(peak, live)
    return peak


@pytest.mark.parametrize("slots,budget", [(3, 1 << 30), (5, 3000), (64, 1 << 30), (2, 1500)])
def test_native_scheduler_feeds_every_packet_once_in_stream_order(slots, budget):
    """The native loop (oasm_replay_ops) against a fake library on the CPU:
    every stream opened, fed exactly its packets in order, ended and closed;
    never more streams open than slots."""
    tr = W.served(seed=3, n_streams=12, n_sig=4, gbps=1.0, duration=0.004, life=0.4)
    fake = NativeFake(slots)
    rc, done, st = native_replay(tr, fake, budget)
    assert rc == 0
    got = sorted(e[2] for e in fake.log if e[0] == "close")
    assert got == sorted(bytes(t) for t in tr.stream_texts() if t.size)
    assert st["packets"] == tr.n_packets and st["bytes"] == int(tr.lens.sum())
    assert st["streams_admitted"] == sum(1 for t in tr.stream_texts() if t.size)
    assert np.isfinite(done).all()
    assert peak_open(fake.log) <= slots
    if slots < 12:
        assert st["max_waiting_streams"] > 0


def test_native_scheduler_waits_out_admission_refused_by_memory():
    """Host fault injection in the native loop: admission refused for memory
    while slots are free; streams wait and every packet is still fed once,
    in order."""
    tr = W.served(seed=5, n_streams=10, n_sig=4, gbps=1.0, duration=0.004, life=0.4)
    fake = NativeFake(slots=8, mem_streams=3)
    rc, done, st = native_replay(tr, fake, 4000)
    assert rc == 0
    got = sorted(e[2] for e in fake.log if e[0] == "close")
    assert got == sorted(bytes(t) for t in tr.stream_texts() if t.size)
    assert st["max_waiting_streams"] > 0
    assert peak_open(fake.log) <= 3


def test_native_scheduler_reports_no_admission_possible():
    """No stream fits the memory budget at all: OASM_ENOMEM, not a hang."""
    tr = W.served(seed=7, n_streams=4, n_sig=4, gbps=1.0, duration=0.002, life=0.4)
    rc, _, _ = native_replay(tr, NativeFake(slots=4, mem_streams=0), 4000)
    assert rc == -2


def test_native_scheduler_surfaces_a_failed_step():
    """Host fault injection in the native loop: a step whose end reports a
    device-wait timeout ends the replay with that error at once."""
    tr = W.served(seed=6, n_streams=6, n_sig=4, gbps=1.0, duration=0.004, life=0.4)
    fake = NativeFake(6, fail_step=3)
    rc, _, _ = native_replay(tr, fake, 2000)
    assert rc == NativeFake.OASM_ETIMEOUT
    assert fake.steps == 3


@pytest.mark.gpu
@pytest.mark.parametrize("slots,budget,realtime,engine",
                         [(4096, 1 << 30, False, "python"), (24, 20000, False, "python"),
                          (64, 1 << 30, True, "python"), (4096, 1 << 30, False, "native"),
                          (24, 20000, False, "native"), (64, 1 << 30, True, "native"),
                          (5, 3000, False, "native"), (4096, 1 << 30, False, "native+zc"),
                          (24, 20000, True, "python+zc")])
def test_served_streams_match_oracle_alone_and_in_the_mix(slots, budget, realtime, engine):
    from parity_util import canon, oracle_rows
    from paper_1712_03560_gb300 import binding as B
    tr = W.served(seed=7, n_streams=48, n_sig=40, mlo=8, mhi=64, gbps=0.2, duration=0.05,
                  life=0.5, planted_frac=0.05)
    with serve.Server(tr.patterns, tr.ks, max_streams=slots, max_batch_bytes=budget) as srv:
        res = srv.replay(tr, realtime=realtime, collect=True, engine=engine.split("+")[0],
                         zero_copy=engine.endswith("+zc"))
    texts = tr.stream_texts()
    assert res["steps"] >= (2 if budget < (1 << 30) or realtime else 1)
    assert res["packets"] == tr.n_packets and res["fed_bytes"] == int(tr.lens.sum())
    if slots < 48:
        assert res["max_waiting_streams"] > 0
    some = 0
    for ext, t in enumerate(texts):
        got = res["hits"].get(ext)
        rows = [] if got is None else [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]),
                                        int(r["start"]), int(r["len"])) for r in got]
        want = oracle_rows(tr.patterns, tr.ks, t)
        assert canon(rows) == want, ext
        some += len(want)
        if ext < 6:  # the same stream alone
            with B.Matcher(tr.patterns, tr.ks) as mt:
                alone = mt.search(t)
            assert canon([(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]),
                           int(r["start"]), int(r["len"])) for r in alone]) == want
    assert some > 0


@pytest.mark.gpu
@pytest.mark.parametrize("engine", ["python", "native"])
def test_served_streams_under_edit_costs_match_oracle(engine):
    """The serving loop on the weighted path: every stream's kept hits equal
    the oracle's under the same edit costs."""
    from parity_util import canon, oracle_rows
    costs = (2, 1, 1)
    tr = W.served(seed=8, n_streams=32, n_sig=24, mlo=8, mhi=64, gbps=0.2, duration=0.04,
                  life=0.5, planted_frac=0.05)
    with serve.Server(tr.patterns, tr.ks, max_streams=16, max_batch_bytes=20000,
                      costs=costs) as srv:
        res = srv.replay(tr, realtime=False, collect=True, engine=engine)
    assert res["packets"] == tr.n_packets and res["steps"] >= 2
    some = 0
    for ext, t in enumerate(tr.stream_texts()):
        got = res["hits"].get(ext)
        rows = [] if got is None else [(int(r["pattern_id"]), int(r["decided_at"]), int(r["k"]),
                                        int(r["start"]), int(r["len"])) for r in got]
        want = oracle_rows(tr.patterns, tr.ks, t, costs=costs)
        assert canon(rows) == want, ext
        some += len(want)
    assert some > 0
