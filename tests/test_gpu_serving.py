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
