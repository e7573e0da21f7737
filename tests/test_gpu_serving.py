"""Serving with continuous batching (needs a GPU).

Every request's result must be identical whether it runs alone or in a mix of requests that
arrive together and overlap on the device, and must equal the direct path on the same database
slice and the oracle on that genome subset.  The device-side input drawer must reproduce the
host drawer byte for byte.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def db():
    import torch

    import __graft_entry__
    import synth.gpu as sg

    __graft_entry__.build()
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Engine

    wl = sg.serving_db(n_genomes=120, median=3e5)
    eng = Engine(0)
    batch = eng.pack_device(wl.d_seq.data_ptr(), wl.offsets.astype(np.uint64))
    ah.ah_ctx_synchronize(eng.ctx)
    torch.cuda.synchronize()
    yield wl, eng, batch
    ah.ah_batch_free(batch)
    eng.close()


def _requests(wl, n, seed=5):
    st = synth.Stream(synth.make_key(seed, 321, 0))
    reqs = []
    for _ in range(n):
        pairs = st.randint(1, 4)
        fwd = [synth.random_primer(st, st.randint(10, 14), st.randint(0, 3), 2) for _ in range(pairs)]
        rev = [synth.random_primer(st, st.randint(10, 14), st.randint(0, 3), 2) for _ in range(pairs)]
        k = [st.randint(0, 2) for _ in range(pairs)]
        count = st.randint(1, wl.n_records)
        first = st.randint(0, wl.n_records - count)
        reqs.append(dict(fwd=fwd, rev=rev, k=k, clamp=2, first_record=first, n_records=count, min_len=30,
                         max_len=3000, orient_mask=15, trim=bool(st.randint(0, 1)), fb_len=6, rb_len=7))
    return reqs


def _key(r):
    return (r["hits"].tobytes(), r["amps"].tobytes(), r["arena"] or b"")


def test_alone_equals_mix(db):
    from paper_2511_00170_gb300 import ah

    wl, eng, batch = db
    reqs = _requests(wl, 10)
    srv = ah.ah_server_create(batch, n_slots=4)
    try:
        alone = []
        for r in reqs:
            alone.append(ah.ah_server_wait(srv, ah.ah_server_submit(srv, **r)))
        tickets = [ah.ah_server_submit(srv, **r) for r in reqs]
        mixed = [ah.ah_server_wait(srv, t) for t in tickets]
    finally:
        ah.ah_server_destroy(srv)
    assert sum(len(x["hits"]) for x in alone) > 0 and sum(len(x["amps"]) for x in alone) > 0
    for a, m in zip(alone, mixed):
        assert _key(a) == _key(m)
    # the mix ran concurrently: some request was admitted before an earlier one finished
    spans = sorted((m["t_admit"], m["t_done"]) for m in mixed)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


@pytest.mark.parametrize("scan_mode", [2, 1, 0])
def test_request_matches_slice_and_oracle(db, scan_mode):
    """Each scan mode (generic while compiling, generic only, generated only) gives the oracle's
    outputs and those of the direct path on a slice of the database."""
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Output, Params

    wl, eng, batch = db
    srv = ah.ah_server_create(batch, n_slots=2)
    ah.ah_server_set_scan_mode(srv, scan_mode)
    try:
        for r in _requests(wl, 3, seed=9 + 10 * scan_mode):
            got = ah.ah_server_wait(srv, ah.ah_server_submit(srv, **r))
            sub = wl.host_subset(range(r["first_record"], r["first_record"] + r["n_records"]))
            sub.fwd, sub.rev, sub.k, sub.clamp = r["fwd"], r["rev"], r["k"], r["clamp"]
            sub.min_len, sub.max_len, sub.trim, sub.fb_len, sub.rb_len = 30, 3000, r["trim"], 6, 7
            ref = oracle.run(sub)
            h, a = got["hits"].copy(), got["amps"].copy()
            h["record"] -= r["first_record"]
            a["record"] -= r["first_record"]
            out = Output(h, a, got["arena"], got["field_off"])
            compare.assert_same_hits(out, ref)
            compare.assert_same_amplicons(out, ref, filtered=False)
            compare.assert_same_sequences(out, ref)
            # and the direct path on a slice of the database
            sl = ah.ah_batch_slice(eng.ctx, batch, r["first_record"], r["n_records"])
            try:
                p = Params(r["fwd"], r["rev"], r["k"], r["clamp"], 30, 3000, 15, trim=r["trim"], fb_len=6, rb_len=7)
                direct = eng.step(sl, p)
            finally:
                ah.ah_batch_free(sl)
            assert direct.hits.tobytes() == h.tobytes() and direct.amps.tobytes() == a.tobytes()
    finally:
        ah.ah_server_destroy(srv)


def test_device_drawer_matches_host_drawer():
    import synth.gpu as sg

    host = synth.batched(n_genomes=24, len_lo=2e3, len_hi=2e5, n_pairs=3)
    dev = sg.batched(n_genomes=24, len_lo=2e3, len_hi=2e5, n_pairs=3)
    assert np.array_equal(host.offsets, dev.offsets)
    assert host.fwd == dev.fwd and host.rev == dev.rev
    assert np.array_equal(host.seq, dev.d_seq.cpu().numpy())


def test_device_dense_drawer_matches_host_drawer():
    """The dense-hit workload drawn on the device (tandem repeats merged where they overlap) equals
    the host drawer byte for byte."""
    import synth.gpu as sg

    host = synth.dense(n_genomes=40, median=1.5e5, sigma=0.3)
    dev = sg.dense(n_genomes=40, median=1.5e5, sigma=0.3)
    assert np.array_equal(host.offsets, dev.offsets)
    assert host.fwd == dev.fwd and host.rev == dev.rev
    assert np.array_equal(host.seq, dev.d_seq.cpu().numpy())


def _large(wl, n_pairs, seed):
    """A request over the whole database with several pairs (a long run on the generic scan)."""
    st = synth.Stream(synth.make_key(seed, 323, 0))
    fwd = [synth.random_primer(st, st.randint(12, 16), st.randint(0, 3), 2) for _ in range(n_pairs)]
    rev = [synth.random_primer(st, st.randint(12, 16), st.randint(0, 3), 2) for _ in range(n_pairs)]
    return dict(fwd=fwd, rev=rev, k=[2] * n_pairs, clamp=2, first_record=0, n_records=wl.n_records, min_len=30,
                max_len=3000, orient_mask=15, trim=False, fb_len=0, rb_len=0)


def test_admission_passes_over_a_request_that_does_not_fit(db):
    """Budget for one large request and one small one beside it.  Two large requests and then small
    ones arrive together: the second large one waits for memory, the small ones are admitted beside
    the first (not held behind the second), the second runs once the first has left, and every
    result equals the request's result alone."""
    from paper_2511_00170_gb300 import ah

    wl, eng, batch = db
    large = [_large(wl, 8, 1), _large(wl, 8, 2)]
    small = [dict(r, first_record=r["first_record"], n_records=1) for r in _requests(wl, 4, seed=21)]
    srv = ah.ah_server_create(batch, n_slots=4)
    ah.ah_server_set_scan_mode(srv, 1)   # no compiles: the large requests run long on the generic scan
    try:
        b_large = max(ah.ah_server_request_bytes(srv, **r) for r in large)
        b_small = max(ah.ah_server_request_bytes(srv, **r) for r in small)
        alone = [ah.ah_server_wait(srv, ah.ah_server_submit(srv, **r)) for r in large + small]
    finally:
        ah.ah_server_destroy(srv)
    # one large and one small fit; two large, or one large and two small, do not
    assert b_large > b_small
    budget = b_large + b_small + (b_large - b_small) // 2
    srv = ah.ah_server_create(batch, n_slots=4, memory_budget=budget)
    ah.ah_server_set_scan_mode(srv, 1)
    try:
        tickets = [ah.ah_server_submit(srv, **r) for r in large + small]
        mixed = [ah.ah_server_wait(srv, t) for t in tickets]
        mem = ah.ah_server_memory(srv)
    finally:
        ah.ah_server_destroy(srv)
    for a, m in zip(alone, mixed):
        assert _key(a) == _key(m)
    l1, l2, smalls = mixed[0], mixed[1], mixed[2:]
    assert l2["t_admit"] >= l1["t_done"] or l1["t_admit"] >= l2["t_done"], "two large requests ran together"
    first = l1 if l1["t_admit"] <= l2["t_admit"] else l2
    second = l2 if first is l1 else l1
    # small requests went ahead of the waiting large one, beside the running one
    assert any(s["t_admit"] < second["t_admit"] and s["t_admit"] < first["t_done"] for s in smalls)
    assert mem["budget"] == budget and mem["reserved"] == 0


def test_injected_allocation_failure_fails_one_request(db):
    """An allocation failure injected on the host fails exactly the request that meets it, with
    AH_ENOMEM; the server goes on serving the others, whose results are unchanged."""
    from paper_2511_00170_gb300 import ah

    wl, eng, batch = db
    reqs = _requests(wl, 4, seed=31)
    srv = ah.ah_server_create(batch, n_slots=1)
    try:
        alone = [ah.ah_server_wait(srv, ah.ah_server_submit(srv, **r)) for r in reqs]
        ah.ah_server_inject_alloc_failures(srv, 1)
        tickets = [ah.ah_server_submit(srv, **r) for r in reqs]
        got, failed = [], 0
        for t in tickets:
            try:
                got.append(ah.ah_server_wait(srv, t))
            except ah.AhError as e:
                assert e.status == ah.AH_ENOMEM and "injected" in str(e)
                failed += 1
                got.append(None)
        again = [ah.ah_server_wait(srv, ah.ah_server_submit(srv, **r)) for r in reqs]
    finally:
        ah.ah_server_destroy(srv)
    assert failed == 1 and got[0] is None   # one slot: the first admitted is the first submitted
    for a, g, b in zip(alone, got, again):
        assert _key(a) == _key(b)
        if g is not None:
            assert _key(a) == _key(g)


def test_cancel_queued_request(db):
    """One slot, a long request running and three queued: the cancelled one finishes with
    AH_ECANCELED without running, the others give their results alone."""
    from paper_2511_00170_gb300 import ah

    wl, eng, batch = db
    long_r = _large(wl, 8, 3)
    reqs = _requests(wl, 3, seed=41)
    srv = ah.ah_server_create(batch, n_slots=1)
    ah.ah_server_set_scan_mode(srv, 1)
    try:
        alone = [ah.ah_server_wait(srv, ah.ah_server_submit(srv, **r)) for r in [long_r] + reqs]
        tickets = [ah.ah_server_submit(srv, **r) for r in [long_r] + reqs]
        ah.ah_server_cancel(srv, tickets[2])
        res = []
        for t in tickets:
            try:
                res.append(ah.ah_server_wait(srv, t))
            except ah.AhError as e:
                res.append(e.status)
        with pytest.raises(ah.AhError):
            ah.ah_server_cancel(srv, tickets[2])   # collected: unknown now
    finally:
        ah.ah_server_destroy(srv)
    assert res[2] == ah.AH_ECANCELED
    for i in (0, 1, 3):
        assert _key(res[i]) == _key(alone[i])


def test_context_allocation_failure_leaves_context_usable(db):
    """A context whose next device allocation is made to fail returns AH_ENOMEM from the call that
    meets it; the same context then runs the step with the same result as before."""
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl, eng, batch = db
    r = _requests(wl, 1, seed=51)[0]
    p = Params(r["fwd"], r["rev"], r["k"], r["clamp"], 30, 3000, 15, trim=r["trim"], fb_len=6, rb_len=7)
    before = eng.step(batch, p)
    ah.ah_ctx_inject_alloc_failures(eng.ctx, 1)
    with pytest.raises(ah.AhError) as e:
        eng.step(batch, p)
    assert e.value.status == ah.AH_ENOMEM
    after = eng.step(batch, p)
    assert before.hits.tobytes() == after.hits.tobytes() and before.amps.tobytes() == after.amps.tobytes()
    assert before.arena == after.arena
