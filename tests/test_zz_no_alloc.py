"""nyx_hydro_estdt_noalloc, the allocation-free CFL step, against the plan-based
nyx_hydro_estdt.

Some callers cannot allocate device memory (a framework owns every
allocation, or a latency-critical loop must stay out of the allocator); this
entry point keeps its scratch in a fixed device array instead.  The test
calls it twice in a row through the C ABI, on two different levels, so the
second call also shows that the shared scratch left by the first is reset.
It runs last (file name) and passes alone or after the other tests."""
import numpy as np
import pytest

from paper_1301_4498_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1301_4498_gb300 import hydro as H  # noqa: E402

TOL = 1e-12  # the FP64 parity tolerance of the other tests


def _reference(w, a):
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl)
    lev = H.make_level(plan, w.state, w.grav)
    a_dev = torch.tensor([a], dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.estdt(lev, a_dev, dt)
    torch.cuda.synchronize()
    return plan, lev, dt.item()


def test_noalloc_estdt_matches_plan_estdt_twice():
    w1 = W.uneven_boxes(nbox=512, boxes=list(range(12)), nsteps=1)
    w2 = W.tiled_box(n=64, box=32, nsteps=1)
    plan1, lev1, ref1 = _reference(w1, 1.0 / 51)
    plan2, lev2, ref2 = _reference(w2, 1.0 / 50)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    a = torch.tensor([1.0 / 51, 1.0 / 50], dtype=torch.float64, device="cuda")
    warm = torch.zeros(1, dtype=torch.float64, device="cuda")
    # a warm-up call loads the kernels, then the two calls under test must
    # leave every allocator untouched
    H.estdt_noalloc(w2.level, lev2.current, a[1:2], warm, gamma=w2.gamma, cfl=w2.cfl)
    torch.cuda.synchronize()
    used0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    H.estdt_noalloc(w1.level, lev1.current, a[0:1], out[0:1], gamma=w1.gamma, cfl=w1.cfl)
    H.estdt_noalloc(w2.level, lev2.current, a[1:2], out[1:2], gamma=w2.gamma, cfl=w2.cfl)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == used0
    assert torch.cuda.mem_get_info()[0] == free0
    got = out.cpu().numpy()
    assert abs(got[0] - ref1) <= TOL * ref1, (got[0], ref1)
    assert abs(got[1] - ref2) <= TOL * ref2, (got[1], ref2)
    assert got[0] != got[1]


def test_noalloc_estdt_rejects_non_finite_cell_width():
    spec = W.independent_boxes_level([(2, 2, 2)], float("inf"))
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(H.NyxError) as e:
        H.estdt_noalloc(spec, x, x[0:1], x[1:2])
    assert e.value.code == H.NYX_EINVAL


def test_noalloc_estdt_rejects_too_many_boxes():
    spec = W.independent_boxes_level([(2, 2, 2)] * (H.NOALLOC_MAX_BOXES + 1), 0.1)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(H.NyxError) as e:
        H.estdt_noalloc(spec, x, x[0:1], x[1:2])
    assert e.value.code == H.NYX_EINVAL
    assert "at most" in str(e.value)
