"""Host-side check of the stream schedules of the box groups, by models of
their enqueue order: a grouped multi-step run (run_grouped in nyx_api.cu)
and, further below, the overlapped host step (step_pipelined).

The run issues, on four streams (the plan stream P, a second advance stream
S2, two fill streams F0, F1):
  * the CFL dt of the first step on P (estdt, with its own finalisation);
    an event on P that both fill streams wait for;
  * per step s (state buffer X = s % 2 read, Y = the other written), per
    group g in the groups' processing order, on fill stream F[gi & 1]: waits
    on the step s-1 advance events of the groups g's fill reads and of g
    itself (s > 0), the ghost fill of g (reads the valid cells of the source
    groups in X, writes g's ghost cells in X), an event;
  * a flattening plan: both fill streams joined into P, then the coefficient
    pass over the whole level on P (reads every cell of X, writes every
    group's coefficients);
  * the step set-up on P (reads dt_s, writes the step constants), an event
    that S2 waits for;
  * per group on P or S2 in turn: a wait on the group's fill event, the
    advance (reads g's valid and ghost cells in X, the step constants and
    g's coefficients; writes g's valid cells in Y; adds to the dt
    accumulator), an event;
  * S2 joined into P, the dt finalisation on P (reads and resets the
    accumulator, writes dt_{s+1});
  * at the end both fill streams joined into P.
A CUDA stream runs its operations in order, and a wait on an event orders
the next operation after the last one issued before the event's record.  The
test builds that happens-before relation and checks that every pair of
operations that touch the same data, one of them writing, is ordered as in
the sequential program (the order of issue), for random groupings, with and
without flattening; five planted mistakes must each be caught.
"""
import itertools
import random

import pytest


class Model:
    def __init__(self):
        self.ops = []            # (name, reads, writes, atomic)
        self.deps = []           # per op: set of op indices it directly follows
        self.last = {}           # stream -> last op index
        self.pending = {}        # stream -> op indices waited for
        self.events = {}         # event -> op index (or None)

    def op(self, stream, name, reads=(), writes=(), atomic=()):
        # atomic: data the operation updates with atomics, which commute with
        # the other atomic updates of the same data (the advances' dt minimum)
        i = len(self.ops)
        d = set(self.pending.pop(stream, ()))
        if stream in self.last:
            d.add(self.last[stream])
        self.ops.append((name, set(reads), set(writes), set(atomic)))
        self.deps.append(d)
        self.last[stream] = i

    def record(self, ev, stream):
        self.events[ev] = self.last.get(stream)

    def wait(self, stream, ev):
        j = self.events.get(ev)
        if j is not None:
            self.pending.setdefault(stream, set()).add(j)

    def check(self):
        n = len(self.ops)
        before = [set() for _ in range(n)]      # transitive predecessors
        for i in range(n):
            for d in self.deps[i]:
                before[i] |= before[d] | {d}
        bad = []
        for a, b in itertools.combinations(range(n), 2):
            na, ra, wa, xa = self.ops[a]
            nb, rb, wb, xb = self.ops[b]
            touch = (wa & (rb | wb)) | (wb & ra) | (xa & (rb | wb)) | (xb & (ra | wa))
            if touch and a not in before[b]:
                bad.append((na, nb, sorted(touch)[:2]))
        return bad


def run_model(ngrp, src, proc, nsteps, flat, mistake=None):
    m = Model()
    allv = lambda X: {("V", X, g) for g in range(ngrp)}
    allh = lambda X: {("H", X, g) for g in range(ngrp)}
    m.op("P", "estdt", reads=allv(0) | {("acc",)}, writes={("dt", 0), ("acc",)})
    m.record("start", "P")
    for k in (0, 1):
        m.wait(f"F{k}", "start")
    for s in range(nsteps):
        X, Y = s % 2, 1 - s % 2
        for gi, g in enumerate(proc):
            fs = f"F{gi & 1}"
            if s > 0:
                need = set(src[g]) | ({g} if mistake != "no_self" else set())
                for q in sorted(need):
                    m.wait(fs, ("adv", q))
            m.op(fs, f"fill{g}.{s}", reads={("V", X, q) for q in src[g]}, writes={("H", X, g)})
            m.record(("fill", g), fs)
        if flat:
            if mistake != "no_fjoin":
                for k in (0, 1):
                    m.record(("fj", k), f"F{k}")
                    m.wait("P", ("fj", k))
            m.op("P", f"flat.{s}", reads=allv(X) | allh(X),
                 writes={("C", g) for g in range(ngrp)})
        m.op("P", f"setup.{s}", reads={("dt", s)}, writes={("SC",)})
        m.record("setup", "P")
        if mistake != "no_setup_wait":
            m.wait("S2", "setup")
        for gi, g in enumerate(proc):
            st = ("P", "S2")[gi & 1]
            if mistake != "no_fill_wait":
                m.wait(st, ("fill", g))
            reads = {("V", X, g), ("H", X, g), ("SC",)} | ({("C", g)} if flat else set())
            m.op(st, f"adv{g}.{s}", reads=reads, writes={("V", Y, g)}, atomic={("acc",)})
            m.record(("adv", g), st)
        m.record("side", "S2")
        if mistake != "no_side_join":
            m.wait("P", "side")
        m.op("P", f"dtfin.{s}", reads={("acc",)}, writes={("acc",), ("dt", s + 1)})
    for k in (0, 1):
        m.record(("fj", k), f"F{k}")
        m.wait("P", ("fj", k))
    return m


def grouping(rng, ngrp):
    """Random source sets (some groups read only themselves or nothing) and
    the processing order of run_grouped: self-contained groups first."""
    src = []
    for g in range(ngrp):
        kind = rng.random()
        if kind < 0.2:
            src.append(set())
        elif kind < 0.4:
            src.append({g})
        else:
            src.append({g} | set(rng.sample(range(ngrp), rng.randint(1, ngrp))))
    proc = [g for g in range(ngrp) if not (src[g] - {g})] + \
           [g for g in range(ngrp) if src[g] - {g}]
    return src, proc


@pytest.mark.parametrize("flat", [False, True])
@pytest.mark.parametrize("seed", range(12))
def test_schedule_orders_every_conflict(seed, flat):
    rng = random.Random(seed)
    ngrp = rng.randint(2, 9)
    src, proc = grouping(rng, ngrp)
    m = run_model(ngrp, src, proc, nsteps=rng.randint(1, 4), flat=flat)
    assert m.check() == []


@pytest.mark.parametrize("mistake,flat", [("no_fill_wait", False), ("no_setup_wait", False),
                                          ("no_fjoin", True), ("no_self", False),
                                          ("no_side_join", False)])
def test_planted_schedule_mistakes_are_caught(mistake, flat):
    caught = False
    for seed in range(40):
        rng = random.Random(1000 + seed)
        ngrp = rng.randint(2, 9)
        src, proc = grouping(rng, ngrp)
        src[proc[0]] = set()          # a group whose fill reads no other group
        m = run_model(ngrp, src, proc, nsteps=4, flat=flat, mistake=mistake)
        if m.check():
            caught = True
            break
    assert caught, mistake


# ---------------------------------------------------------------------------
# The overlapped host step (step_pipelined in nyx_api.cu, dt given): the
# plan stream P, a second advance stream S2, the input stream IN and the
# read-back stream OUT.  The host buffers may be one buffer (host_in ==
# host_out), and the device staging buffer (packed) serves both directions.

def host_step_model(ngrp, src, proc, in_order, flat, same_host, mistake=None):
    m = Model()
    hin = "host" if same_host else "host_in"
    hout = "host" if same_host else "host_out"
    X, Y = 0, 1
    m.op("P", "scalars", writes={("scal",)})
    m.record("start", "P")
    m.wait("IN", "start")
    for q in in_order:
        m.op("IN", f"copy_in{q}", reads={(hin, q)}, writes={("packed", q)})
        m.op("IN", f"scatter{q}", reads={("packed", q)}, writes={("V", X, q)})
        m.record(("in", q), "IN")
    m.op("P", "setup", reads={("scal",)}, writes={("SC",)})
    m.record("setup", "P")
    m.wait("S2", "setup")
    waited = [set(), set()]
    for gi, g in enumerate(proc):
        st = ("P", "S2")[gi & 1]
        need = (set(src[g]) | {g}) - waited[gi & 1]
        if mistake == "no_own_input":
            need -= {g}
        for q in sorted(need):
            m.wait(st, ("in", q))
        waited[gi & 1] |= need
        m.op(st, f"fill{g}", reads={("V", X, q) for q in src[g]}, writes={("H", X, g)})
        if flat:
            m.op(st, f"flat{g}", reads={("V", X, g), ("H", X, g)}, writes={("C", g)})
        reads = {("V", X, g), ("H", X, g), ("SC",)} | ({("C", g)} if flat else set())
        m.op(st, f"adv{g}", reads=reads, writes={("V", Y, g)}, atomic={("acc",)})
        m.op(st, f"gather{g}", reads={("V", Y, g)}, writes={("packed", g)})
        m.record(("grp", g), st)
        if mistake != "no_out_wait":
            m.wait("OUT", ("grp", g))
        m.op("OUT", f"copy_out{g}", reads={("packed", g)}, writes={(hout, g)})
    m.record("side", "S2")
    m.wait("P", "side")
    m.op("P", "dtfin", reads={("acc",)}, writes={("acc",), ("scal_dt",)})
    return m


def host_step_grouping(rng, ngrp):
    src, proc = grouping(rng, ngrp)
    order, sent = [], set()
    for g in proc:                     # inputs in the order the advances need them
        for q in sorted(set(src[g]) | {g}):
            if q not in sent:
                sent.add(q)
                order.append(q)
    return src, proc, order


@pytest.mark.parametrize("flat,same_host", [(False, False), (True, False), (False, True)])
@pytest.mark.parametrize("seed", range(8))
def test_host_step_schedule_orders_every_conflict(seed, flat, same_host):
    rng = random.Random(500 + seed)
    ngrp = rng.randint(2, 9)
    src, proc, order = host_step_grouping(rng, ngrp)
    assert sorted(order) == list(range(ngrp))
    m = host_step_model(ngrp, src, proc, order, flat, same_host)
    assert m.check() == []


@pytest.mark.parametrize("mistake", ["no_own_input", "no_out_wait"])
def test_planted_host_step_mistakes_are_caught(mistake):
    caught = False
    for seed in range(40):
        rng = random.Random(2000 + seed)
        ngrp = rng.randint(2, 9)
        src, proc, order = host_step_grouping(rng, ngrp)
        src[proc[0]] = set()
        m = host_step_model(ngrp, src, proc, order, False, True, mistake=mistake)
        if m.check():
            caught = True
            break
    assert caught, mistake
