"""Host-side check of the hand-overs between the column threads and the
update warps of the task-form kernel (nyx_fused2.cuh).

The kernel's column threads (producer of fluxes) and update threads
(consumer of fluxes, and producer of each plane's inputs) meet on four named
barriers per box tile:
  * a work item is a tile's planes [zb, ze) (the whole column, zb = 0 and
    ze = nz, or a chunk of it);
  * the update warps write the primitive ring's planes zb-3 .. zb+1 and plane
    zb-1's frame, gravity and flattening rows, and arrive on LOADED; then for
    c = zb .. ze they wait on CONSUMED (and send the tensor copies of plane
    c+1's inputs into the staging buffer that plane c-1 used), write ring
    plane c+2 and plane c's frame, arrive on LOADED, and (c >= zb+2) wait on
    READY, update plane c-2 and arrive on FREE; finally they wait on READY
    and update plane ze-1;
  * the column threads, plane step c = zb-1 .. ze: wait on LOADED, trace
    plane c (ring planes c-2 .. c+2, the frame of plane c), pass their stage
    barrier, arrive on CONSUMED when c < ze, run their other stages, wait on
    FREE when c >= zb+2, store the fluxes of plane c-1 (x/y buffer) and of z
    face c (slot c & 1), and arrive on READY when c >= zb+1;
  * both then meet on the CTA-wide barrier before the next item.
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


def producer_ops(zb, ze):
    ops = []
    for c in range(zb - 1, ze + 1):
        ops.append(("sync", BAR_LOADED, NT))
        ops.append(("trace", c))
        ops.append(("sync", BAR_COL, NTC))           # end of the trace stage
        if c < ze:
            ops.append(("arrive", BAR_CONSUMED, NT))
        ops += [("sync", BAR_COL, NTC)] * 2          # stage barriers after S2 and S3
        if c >= zb + 2:
            ops.append(("sync", BAR_FREE, NT))
        ops.append(("store", c))
        if c >= zb + 1:
            ops.append(("arrive", BAR_READY, NT))
    ops.append(("sync", BAR_ALL, NT))
    return ops


def consumer_ops(zb, ze):
    ops = [("prologue",), ("write", zb - 1), ("arrive", BAR_LOADED, NT)]
    for c in range(zb, ze + 1):
        ops.append(("sync", BAR_CONSUMED, NT))
        ops.append(("write", c))
        ops.append(("arrive", BAR_LOADED, NT))
        if c >= zb + 2:
            ops.append(("sync", BAR_READY, NT))
            ops.append(("load", c - 2))
            ops.append(("arrive", BAR_FREE, NT))
    ops.append(("sync", BAR_READY, NT))
    ops.append(("load", ze - 1))
    ops.append(("sync", BAR_ALL, NT))
    return ops


def _items(depths):
    """Work items (zb, ze): an int is a whole column of that depth, a pair
    a chunk of planes."""
    return [(0, d) if isinstance(d, int) else tuple(d) for d in depths]


def simulate(depths, rng):
    weight = {"P": NTC, "C": NU}
    items = _items(depths)
    prog = {"P": [op for zb, ze in items for op in producer_ops(zb, ze)],
            "C": [op for zb, ze in items for op in consumer_ops(zb, ze)]}
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
            zb = items[t][0]
            for k in range(zb - 3, zb + 1):
                ring[(k + 8) % 5] = (t, k)
        elif op[0] == "write":
            c, t = op[1], tile["C"]
            zb, ze = items[t]
            k = c + 2                                 # ring plane written
            old = ring.get((k + 8) % 5)
            if old is not None and old[0] == t:
                q = old[1]
                for cc in range(max(zb - 1, q - 2), min(ze, q + 2) + 1):
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
            zb = items[t][0]
            if c >= zb + 1:
                assert not xy.get("live"), f"x/y fluxes of plane {xy.get('plane')} overwritten"
                xy.update(tile=t, plane=c - 1, live=True)
            if c >= zb:
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
            if p == items[t][1] - 1:
                zf[(p + 1) & 1]["live"] = False  # the tile's last face


@pytest.mark.parametrize("depths", [[1], [2], [3], [4], [5], [8], [32], [64],
                                    [1, 2, 3, 4, 5, 6, 7, 8], [32, 64, 32, 1, 3],
                                    [(0, 112), (112, 128), (0, 16)],
                                    [(5, 6), (6, 8), (0, 5), (3, 4), (40, 43)],
                                    [(64, 128), 16, (17, 33), (1, 2)]])
def test_flux_handover_protocol(depths):
    for seed in range(200):
        simulate(depths, random.Random(seed))


def test_planted_input_mistake_is_caught():
    """Update warps that write the next plane's inputs without waiting for
    the trace of the previous plane must fail."""
    global consumer_ops
    saved = consumer_ops

    def eager(zb, ze):
        ops = saved(zb, ze)
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

    def early(zb, ze):
        ops = saved(zb, ze)
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
