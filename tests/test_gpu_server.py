"""The serving loop (wl_server_*): requests for different lattices admitted by
their device footprint against a memory budget, walked concurrently on the
GPU, and each result identical to the same request run alone."""
import numpy as np
import pytest

import paper_1302_2320_gb300 as wl

pytestmark = pytest.mark.gpu

REQUESTS = [("square", 8, 3), ("square", 6, 5), ("triangular", 6, 7), ("cubic", 4, 9),
            ("square", 12, 1), ("square", 8, 4), ("triangular", 5, 2), ("square", 10, 6)]
U, C, BUDGET = 1e-6, 1000, 1_500_000


def solo(lattice, L, seed):
    h = wl.Handle(lattice, L, seed=seed, check_interval=C, move_budget=BUDGET)
    h.run(U, 0.8)
    h.assemble()
    surf, _ = h.get_surface()
    h.close()
    return surf


def test_mixed_requests_match_solo_runs_and_overlap():
    sizes = [wl.wl_required_bytes(wl.LATTICES[lat], L) for lat, L, _ in REQUESTS]
    budget = sorted(sizes)[-1] + sorted(sizes)[-2]          # room for two large at a time
    srv = wl.Server(hbm_budget=budget, max_active=4)
    ids = [srv.submit(lat, L, seed=seed, ln_f_min=U, check_interval=C, move_budget=BUDGET)
           for lat, L, seed in REQUESTS]
    for rid in ids:
        assert srv.wait(rid, 300.0) in (wl.WL_OK, wl.WL_ENOTCONVERGED)
    infos = [srv.info(rid) for rid in ids]
    for (lat, L, seed), rid, info in zip(REQUESTS, ids, infos):
        assert info["state"] == 2
        assert info["submit_s"] <= info["start_s"] <= info["finish_s"]
        got = srv.result(rid)
        assert np.array_equal(got, solo(lat, L, seed)), (lat, L, seed)
        srv.release(rid)
    # continuous batching: some requests ran at the same time ...
    spans = [(i["start_s"], i["finish_s"], i["device_bytes"]) for i in infos]
    overlaps = [(a, b) for x, a in enumerate(spans) for b in spans[x + 1:]
                if a[0] < b[1] and b[0] < a[1]]
    assert overlaps
    # ... and the admitted ones never held more than the budget together
    for t in sorted(s for s, _, _ in spans):
        held = sum(b for s, f, b in spans if s <= t < f)
        assert held <= budget
    srv.close()


def test_request_larger_than_budget_is_refused():
    srv = wl.Server(hbm_budget=1 << 20, max_active=2)
    with pytest.raises(wl.WLError) as e:
        srv.submit("square", 64)
    assert e.value.status == 2                             # WL_ENOMEM
    srv.close()


def test_pooled_handles_are_reused_and_evicted():
    """Requests of one lattice reuse a finished request's handle (same results
    as solo runs); with room for one handle at a time, alternating lattices
    evict the idle handle of the other lattice and still complete."""
    reqs = [("square", 10, 11), ("square", 10, 12), ("triangular", 6, 13), ("square", 10, 14),
            ("triangular", 6, 15)]
    budget = max(wl.wl_required_bytes(wl.LATTICES[lat], L) for lat, L, _ in reqs)
    srv = wl.Server(hbm_budget=budget, max_active=2)
    ids = [srv.submit(lat, L, seed=seed, ln_f_min=U, check_interval=C, move_budget=300_000)
           for lat, L, seed in reqs]
    for rid, (lat, L, seed) in zip(ids, reqs):
        assert srv.wait(rid, 300.0) in (wl.WL_OK, wl.WL_ENOTCONVERGED)
        h = wl.Handle(lat, L, seed=seed, check_interval=C, move_budget=300_000)
        h.run(U, 0.8)
        h.assemble()
        ref, _ = h.get_surface()
        h.close()
        assert np.array_equal(srv.result(rid), ref), (lat, L, seed)
    infos = [srv.info(rid) for rid in ids]
    spans = sorted((i["start_s"], i["finish_s"]) for i in infos)
    for a, b in zip(spans, spans[1:]):
        assert b[0] >= a[1] - 1e-9           # one handle's room: never two at once
    srv.close()
