"""Host-side check of the hand-overs between the column threads and the
update warps of the task-form kernel (nyx_fused2.cuh).

The kernel's column threads (producer of fluxes) and update threads
(consumer of fluxes, and producer of each plane's inputs) meet on four named
barriers per box tile:
  * the update warps write the primitive ring's planes -3 .. 1 and plane -1's
    frame, gravity and flattening rows, and arrive on LOADED; then for
    c = 0 .. nz they wait on CONSUMED, write ring plane c+2 and plane c's
    frame, arrive on LOADED, and (c >= 2) wait on READY, update plane c-2
    and arrive on FREE when c <= nz; finally they wait on READY and update
    plane nz-1;
  * the column threads, plane step c = -1 .. nz: wait on LOADED, trace plane
    c (ring planes c-2 .. c+2, the frame of plane c), pass their stage
    barrier, arrive on CONSUMED when c < nz, run their other stages, wait on
    FREE when c >= 2, store the fluxes of plane c-1 (x/y buffer) and of z
    face c (slot c & 1), and arrive on READY when c >= 1;
  * both then meet on the CTA-wide barrier before the next tile.
This test models bar.sync / bar.arrive phase counting (a phase completes when
the arrivals reach the barrier's thread count) and runs the two sequences
under random interleavings.  It checks that every phase completes with exactly
one producer and one consumer arrival, that nothing deadlocks, that the
consumer reads only fluxes that were stored for its plane, and that no buffer
is overwritten while a plane that needs it is not yet updated.
"""
import random

import pytest

NTC, NU = 576, 128          # 16x8 tile: 3 x 192 column threads, 4 update warps
NT = NTC + NU
BAR_ALL, BAR_COL, BAR_READY, BAR_FREE, BAR_LOADED, BAR_CONSUMED = 0, 1, 2, 3, 4, 5


def producer_ops(nz):
    ops = []
    for c in range(-1, nz + 1):
        ops.append(("sync", BAR_LOADED, NT))
        ops.append(("trace", c))
        ops.append(("sync", BAR_COL, NTC))           # end of the trace stage
        if c < nz:
            ops.append(("arrive", BAR_CONSUMED, NT))
        ops += [("sync", BAR_COL, NTC)] * 4          # stage barriers S2..S5
        if c >= 2:
            ops.append(("sync", BAR_FREE, NT))
        ops.append(("store", c))
        if c >= 1:
            ops.append(("arrive", BAR_READY, NT))
    ops.append(("sync", BAR_ALL, NT))
    return ops


def consumer_ops(nz):
    ops = [("prologue",), ("write", -1), ("arrive", BAR_LOADED, NT)]
    for c in range(0, nz + 1):
        ops.append(("sync", BAR_CONSUMED, NT))
        ops.append(("write", c))
        ops.append(("arrive", BAR_LOADED, NT))
        if c >= 2:
            ops.append(("sync", BAR_READY, NT))
            ops.append(("load", c - 2))
            if c <= nz:
                ops.append(("arrive", BAR_FREE, NT))
    ops.append(("sync", BAR_READY, NT))
    ops.append(("load", nz - 1))
    ops.append(("sync", BAR_ALL, NT))
    return ops


def simulate(depths, rng):
    weight = {"P": NTC, "C": NU}
    prog = {"P": [op for nz in depths for op in producer_ops(nz)],
            "C": [op for nz in depths for op in consumer_ops(nz)]}
    pos = {"P": 0, "C": 0}
    tile = {"P": 0, "C": 0}
    bars = {}
    blocked = {}
    xy = {}        # the single x/y buffer: (tile, plane, live)
    zf = {}        # z-face slots: slot -> (tile, face, live)
    ring = {}      # primitive ring: slot (plane + 8) % 5 -> (tile, plane)
    frame = {}     # the framed plane (with gravity and flattening rows): (tile, plane)
    traced = set()  # (tile, plane) traced by the column threads
    steps = 0
    while True:
        steps += 1
        assert steps < 10 ** 6
        ready = [a for a in "PC" if a not in blocked and pos[a] < len(prog[a])]
        if not ready:
            assert not blocked, f"deadlock: {blocked}"
            return
        a = rng.choice(ready)
        op = prog[a][pos[a]]
        pos[a] += 1
        if op[0] in ("sync", "arrive"):
            _, bid, limit = op
            b = bars.setdefault(bid, {"count": 0, "who": [], "waiting": []})
            b["count"] += weight[a]
            b["who"].append(a)
            assert b["count"] <= limit, f"barrier {bid} overflows: {b['who']}"
            if op[0] == "sync":
                b["waiting"].append(a)
                blocked[a] = bid
            if b["count"] == limit:
                expect = ["P"] if limit == NTC else ["C", "P"]
                assert sorted(b["who"]) == expect, f"barrier {bid} phase by {b['who']}"
                for x in b["waiting"]:
                    blocked.pop(x, None)
                bars[bid] = {"count": 0, "who": [], "waiting": []}
                if bid == BAR_ALL:
                    tile["P"] += 1
                    tile["C"] += 1
        elif op[0] == "prologue":
            t = tile["C"]
            for k in range(-3, 1):
                ring[(k + 8) % 5] = (t, k)
        elif op[0] == "write":
            c, t = op[1], tile["C"]
            nz = depths[t]
            k = c + 2                                 # ring plane written
            old = ring.get((k + 8) % 5)
            if old is not None and old[0] == t:
                q = old[1]
                for cc in range(max(-1, q - 2), min(nz, q + 2) + 1):
                    assert (t, cc) in traced, f"ring plane {q} overwritten before trace {cc}"
            ring[(k + 8) % 5] = (t, k)
            if frame and frame["tile"] == t:
                assert (t, frame["plane"]) in traced, f"frame {frame['plane']} overwritten"
            frame.update(tile=t, plane=c)
        elif op[0] == "trace":
            c, t = op[1], tile["P"]
            for k in range(c - 2, c + 3):
                assert ring.get((k + 8) % 5) == (t, k), f"trace {c}: ring plane {k} missing"
            assert frame.get("tile") == t and frame.get("plane") == c, f"trace {c}: frame"
            traced.add((t, c))
        elif op[0] == "store":
            c, t = op[1], tile["P"]
            if c >= 1:
                assert not xy.get("live"), f"x/y fluxes of plane {xy.get('plane')} overwritten"
                xy.update(tile=t, plane=c - 1, live=True)
            if c >= 0:
                old = zf.get(c & 1)
                assert not (old and old["live"]), f"z face {old and old['face']} overwritten"
                zf[c & 1] = {"tile": t, "face": c, "live": True}
        else:
            p, t = op[1], tile["C"]
            assert xy.get("live") and (xy["tile"], xy["plane"]) == (t, p)
            for f in (p, p + 1):
                s = zf.get(f & 1)
                assert s and s["live"] and (s["tile"], s["face"]) == (t, f)
            xy["live"] = False
            zf[p & 1]["live"] = False           # face p is needed by plane p only from now on
            nz = depths[t]
            if p == nz - 1:
                zf[(p + 1) & 1]["live"] = False  # the tile's last face


@pytest.mark.parametrize("depths", [[1], [2], [3], [4], [5], [8], [32], [64],
                                    [1, 2, 3, 4, 5, 6, 7, 8], [32, 64, 32, 1, 3]])
def test_flux_handover_protocol(depths):
    for seed in range(200):
        simulate(depths, random.Random(seed))


def test_planted_input_mistake_is_caught():
    """Update warps that write the next plane's inputs without waiting for
    the trace of the previous plane must fail."""
    global consumer_ops
    saved = consumer_ops

    def eager(nz):
        ops = saved(nz)
        for i in range(len(ops) - 1):       # write before the wait, counts unchanged
            if ops[i][:2] == ("sync", BAR_CONSUMED) and ops[i + 1][0] == "write":
                ops[i], ops[i + 1] = ops[i + 1], ops[i]
        return ops

    consumer_ops = eager
    try:
        caught = 0
        for seed in range(200):
            try:
                simulate([8], random.Random(seed))
            except AssertionError:
                caught += 1
        assert caught > 0
    finally:
        consumer_ops = saved


def test_planted_protocol_mistake_is_caught():
    """A consumer that releases its buffers one plane early must fail."""
    global consumer_ops
    saved = consumer_ops

    def early(nz):
        ops = saved(nz)
        out = []
        for op in ops:
            if op[0] == "load":
                # arrive on FREE before the load instead of after it
                nxt = ops[ops.index(op) + 1] if ops.index(op) + 1 < len(ops) else None
                if nxt is not None and nxt[0] == "arrive":
                    out.append(nxt)
                out.append(op)
            elif op[0] == "arrive" and out and out[-1][0] == "load":
                continue
            else:
                out.append(op)
        return out

    consumer_ops = early
    try:
        caught = 0
        for seed in range(200):
            try:
                simulate([8], random.Random(seed))
            except AssertionError:
                caught += 1
        assert caught > 0
    finally:
        consumer_ops = saved
