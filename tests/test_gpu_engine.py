"""The batched inpainting engine (hdi_engine_*, and hdi_inpaint_batch on top
of it): images of uneven size in one launch per solver phase, each stopping
at its own tolerance, admitted by the engine's real workspace bytes and
joining at V-cycle boundaries. Results are checked against the FP64 oracle
(Sec. 2.1) and against the single-image solve."""

import numpy as np
import pytest

from gpu_util import torch, need_gpu, ctx, dev
from oracle import inpaint as inpaint_ref, rel_residual
from synthdata import synth_image, synth_rgb, random_mask

pytestmark = pytest.mark.gpu

SHAPES = [(96, 128, 3, 0.04), (64, 64, 1, 0.08), (50, 70, 1, 0.02), (160, 96, 3, 0.01), (33, 33, 1, 0.1),
          (1, 40, 1, 0.2), (130, 77, 3, 0.05), (20, 300, 1, 0.03)]


def make(i, H, W, ch, d):
    f = synth_rgb(H, W, seeds=(i, i + 100, i + 200)) if ch == 3 else synth_image(H, W, i + 300)[None]
    return f.astype(np.float32), random_mask(H, W, d, i + 400)


def engine(**kw):
    import paper_2401_06747_b300 as hdi
    return hdi.Engine(0, **kw)


def test_engine_uneven_sizes_against_oracle_and_single_solves():
    need_gpu()
    data = [make(i, *s) for i, s in enumerate(SHAPES)]
    e = engine(budget_gb=4.0)
    outs = []
    for i, (f, c) in enumerate(data):
        o = torch.empty((f.shape[0],) + f.shape[1:], dtype=torch.float32, device="cuda")
        assert e.submit(dev(f), dev(c), o, tol=1e-6, tag=i)
        outs.append(o)
    assert e.status()["in_flight"] == len(data)
    done = {}
    steps = 0
    while len(done) < len(data):
        for tag, st in e.step():
            done[tag] = st
        steps += 1
        assert steps < 100
    assert e.status()["in_flight"] == 0 and e.status()["bytes_in_use"] == 0
    k = ctx()
    for i, ((f, c), o) in enumerate(zip(data, outs)):
        st = done[i]
        assert st["status"] == 0 and st["rel_res"] <= 1e-6
        u = o.cpu().numpy().astype(np.float64)
        f64 = f.astype(np.float64)
        assert rel_residual(u, f64, c).max() <= 1.5e-6
        assert np.abs(u - inpaint_ref(f64, c)).max() <= 1e-3
        single = torch.empty_like(o)
        s1 = k.inpaint(dev(f), dev(c), single, tol=1e-6)
        assert (single - o).abs().max().item() <= 1e-3
        # the refinement steps of the image solved alone (the norms are summed
        # in another order, which may move a borderline stop by one step)
        assert abs(st["iterations"] - s1["iterations"]) <= 1, (i, st, s1)


def test_launches_do_not_grow_with_the_number_of_images():
    """One launch per solver phase: eight images of eight sizes take about as
    many batched launches as the slowest image alone."""
    need_gpu()
    data = [make(i, *s) for i, s in enumerate(SHAPES)]

    def run(items):
        e = engine(budget_gb=4.0)
        outs = []
        for i, (f, c) in enumerate(items):
            o = torch.empty_like(dev(f))
            assert e.submit(dev(f), dev(c), o, tol=1e-6, tag=i)
            outs.append(o)
        n = 0
        while n < len(items):
            n += len(e.step())
        return e.launch_count()

    all_launches = run(data)
    singles = [run([d]) for d in data]
    # eight images of eight sizes: not eight times the launches (one launch per
    # phase), only the extra FMG starts of hierarchies ending at other levels
    # and the steps of the image that needs the most V-cycles
    assert all_launches <= 1.5 * max(singles), (all_launches, singles)
    assert all_launches <= sum(singles) / 3, (all_launches, singles)


def test_admission_by_workspace_and_joins_between_steps():
    """A budget that holds two requests: a third is refused until one
    finishes; a request submitted while others are in their V-cycles gets the
    same result as alone."""
    need_gpu()
    import paper_2401_06747_b300 as hdi
    H, W = 200, 240
    per = hdi.Engine.request_bytes(H, W, 3)
    assert per > 0
    e = engine(budget_gb=2.5 * per / 1e9)
    items = [make(10 + i, H, W, 3, 0.03 + 0.01 * i) for i in range(4)]
    outs = [torch.empty_like(dev(f)) for f, _ in items]
    assert e.submit(dev(items[0][0]), dev(items[0][1]), outs[0], tol=1e-7, tag=0)
    assert e.submit(dev(items[1][0]), dev(items[1][1]), outs[1], tol=1e-7, tag=1)
    assert e.status()["bytes_in_use"] == 2 * per
    assert not e.submit(dev(items[2][0]), dev(items[2][1]), outs[2], tol=1e-7, tag=2)
    assert e.status()["in_flight"] == 2
    done = {}
    pending = [2, 3]
    steps = 0
    while len(done) < 4:
        for tag, st in e.step():
            done[tag] = st
        steps += 1
        # join at the V-cycle boundary as soon as the workspace allows
        while pending and e.submit(dev(items[pending[0]][0]), dev(items[pending[0]][1]), outs[pending[0]],
                                   tol=1e-7, tag=pending[0]):
            pending.pop(0)
        assert e.status()["bytes_in_use"] <= 2 * per
        assert steps < 200
    k = ctx()
    for i, ((f, c), o) in enumerate(zip(items, outs)):
        assert done[i]["status"] == 0
        single = torch.empty_like(o)
        k.inpaint(dev(f), dev(c), single, tol=1e-7)
        assert (single - o).abs().max().item() <= 1e-3
        assert np.abs(o.cpu().numpy().astype(np.float64) - inpaint_ref(f.astype(np.float64), c)).max() <= 1e-3


def test_batch_modes_agree():
    """hdi_inpaint_batch through the engine and through size classes."""
    need_gpu()
    data = [make(i, *s) for i, s in enumerate(SHAPES[:5])] + [make(20, 96, 128, 3, 0.04)]
    fs = [dev(f) for f, _ in data]
    ms = [dev(c) for _, c in data]
    o1 = [torch.empty_like(x) for x in fs]
    o2 = [torch.empty_like(x) for x in fs]
    s1 = ctx(batch_engine=1).inpaint_batch(fs, ms, o1, tol=1e-6)
    s2 = ctx(batch_engine=0).inpaint_batch(fs, ms, o2, tol=1e-6)
    for a, b, x, y in zip(o1, o2, s1, s2):
        assert x["rel_res"] <= 1e-6 and y["rel_res"] <= 1e-6
        assert (a - b).abs().max().item() <= 1e-3


def test_engine_errors():
    need_gpu()
    import paper_2401_06747_b300 as hdi
    e = engine(budget_gb=1.0)
    f = dev(synth_image(16, 16, 1).astype(np.float32)[None])
    o = torch.empty_like(f)
    empty = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(hdi.HdiError) as ei:
        e.submit(f, empty, o, tol=1e-6, tag=0)
    assert ei.value.code == -2
    with pytest.raises(hdi.HdiError) as ei:
        e.submit(f, dev(random_mask(16, 16, 0.1, 2)), o, tol=2.0, tag=0)
    assert ei.value.code == -1
    assert e.status()["bytes_in_use"] == 0
    assert e.step() == []


def test_engine_results_reproducible_bit_for_bit():
    """Engines fed the same requests return the same bits: every norm comes
    from a deterministic segmented reduction whose partials no other
    reduction of the launch overwrites (the first refinement residual sums
    ||r||^2 and ||b||^2 in one launch)."""
    need_gpu()
    import paper_2401_06747_b300 as hdi
    data = [make(i, *s) for i, s in enumerate(SHAPES)] + [make(30, 260, 390, 3, 0.04)]
    ref = None
    for _ in range(5):
        e = hdi.Engine(0, budget_gb=4.0)
        outs = []
        for i, (f, c) in enumerate(data):
            o = torch.empty_like(dev(f))
            assert e.submit(dev(f), dev(c), o, tol=1e-7, tag=i)
            outs.append(o)
        n = 0
        while n < len(data):
            n += len(e.step())
        got = [o.cpu().numpy() for o in outs]
        e.close()
        if ref is None:
            ref = got
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)
