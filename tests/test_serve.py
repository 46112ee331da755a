"""Serving loop: admission by budget (host logic, CPU) and results in the mix
equal to results alone (GPU)."""

import threading

import numpy as np
import pytest

from paper_2401_06747_b300.serve import Budget, tensor_bytes, Request


def test_budget_admission_is_bounded_and_thread_safe():
    b = Budget(1000)
    assert b.try_take(600)
    assert not b.try_take(600)          # would exceed the budget
    assert b.try_take(400)
    b.give(600)
    assert b.try_take(500)
    b.give(400)
    b.give(500)
    assert b.used == 0
    assert b.try_take(5000)             # an oversized request runs alone
    assert not b.try_take(1)
    b.give(5000)
    seen = []

    def worker():
        for _ in range(200):
            if b.try_take(10):
                seen.append(b.used)
                b.give(10)

    ts = [threading.Thread(target=worker) for _ in range(8)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert b.used == 0 and max(seen) <= 1000


def test_tensor_bytes_and_held_workspace():
    f = np.zeros((3, 100, 200), np.float32)
    assert tensor_bytes(f) == 8 * 3 * 100 * 200 + 100 * 200
    b = Budget(1000)
    b.hold(900)                         # workspace already allocated is charged without a check
    assert b.try_take(200)              # nothing but held bytes charged: runs (cannot block the queue)
    assert not b.try_take(50)           # now it does not fit
    b.give(200)
    assert b.try_take(100)


def test_engine_request_bytes_from_the_library():
    """The inpaint charge is the library's own workspace figure for the shape
    (no GPU needed to compute it): it grows with the pixel count and the
    channels."""
    import paper_2401_06747_b300 as hdi
    a = hdi.Engine.request_bytes(100, 200, 1)
    b = hdi.Engine.request_bytes(100, 200, 3)
    c = hdi.Engine.request_bytes(200, 400, 3)
    assert 0 < a < b < c
    assert 40 * 3 * 100 * 200 < b < 80 * 3 * 100 * 200
    assert hdi.Engine.request_bytes(0, 5, 1) == -1


@pytest.mark.gpu
def test_results_in_the_mix_equal_results_alone():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_06747_b300 as hdi
    from paper_2401_06747_b300.serve import Server, densify_to
    from synthdata import synth_rgb, serving_stream, serving_inputs
    base = synth_rgb(300, 400, seeds=(1, 2, 3), dtype=np.float32)
    specs = serving_stream(36, 400.0, 11)
    reqs = []
    for s in specs:
        s = dict(s, height=min(s["height"] // 16, 300), width=min(s["width"] // 16, 400))
        f, m = serving_inputs(s, base)
        reqs.append(Request(id=s["id"], kind=s["kind"], arrival=s["arrival"], f=f, mask=m, density=0.03, seed=s["seed"]))
    reqs[1].kind = "tonal"
    reqs[2].kind = "densify"
    srv = Server(0, budget_gb=1.0, workers=2)
    res = srv.run(reqs)
    assert res["requests"] == len(reqs)
    assert res["engine_steps"] > 0 and res["max_inpaint_in_flight"] >= 2
    alone = hdi.Context(0)
    for r in srv.done:
        fd = torch.from_numpy(r.f).cuda()
        out = torch.empty_like(fd)
        got, gmask = r.result
        if r.kind == "inpaint":
            alone.inpaint(fd, torch.from_numpy(r.mask).cuda(), out, tol=1e-6)
            assert np.abs(out.cpu().numpy() - got).max() <= 1e-3
        elif r.kind == "tonal":
            alone.tonal_opt(fd, torch.from_numpy(r.mask).cuda(), out, tol=1e-6)
            np.testing.assert_array_equal(out.cpu().numpy(), got)
        else:
            md = torch.zeros(r.f.shape[1:], dtype=torch.uint8, device="cuda")
            densify_to(alone, fd, md, out, 0.03, r.seed, 1e-6)
            np.testing.assert_array_equal(md.cpu().numpy(), gmask)
            assert np.abs(out.cpu().numpy() - got).max() <= 1e-3
