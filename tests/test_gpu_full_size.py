"""The path at the workloads' full sizes, in the launch configuration the bench times (needs a GPU).

Each workload is scanned as the bench scans it: one autotuned, graph-captured plan over the whole
batch.  The oracle cannot run the whole batch in a test's time, so it runs seeded samples of
records one by one, and those records' sites, amplicons, Tm and sequences must equal the plan's
output restricted to them (records are independent in every step of the path).  Properties that
hold at any size are checked over the whole output: site order and bounds, mismatch budgets,
amplicon geometry and orientation, and the lengths of every extracted field.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2511_00170_gb300.pipeline import Engine

    e = Engine(0)
    yield e
    e.close()


def _plan_output(engine, batch, p, with_seqs=True):
    """Plan exactly as the bench builds it, one checked run, the results on the host."""
    from paper_2511_00170_gb300 import ah

    plan = engine.plan(batch, p, with_seqs=with_seqs, autotune=True, persistent=-1)
    try:
        ah.ah_plan_run(plan, engine.ctx)
        ah.ah_plan_launch(plan, engine.ctx)   # a replay of the captured graph gives the output read below
        return engine.plan_output(plan, with_seqs=with_seqs), ah.ah_plan_info_get(plan)
    finally:
        ah.ah_plan_free(plan)


def _check_properties(out, wl, lengths):
    """Invariants of the path at any size (readings R6-R12, R17, R18)."""
    h, a = out.hits, out.amps
    plen = np.array([[len(f), len(r)] for f, r in zip(wl.fwd, wl.rev)], dtype=np.int64)
    pat = h["pattern"].astype(np.int64)
    pair, primer, strand = pat >> 2, pat & 1, (pat >> 1) & 1
    L = plen[pair, primer]
    # order (pair, record, pos, orient), unique
    key = np.stack([pair, h["record"].astype(np.int64), h["pos"].astype(np.int64), pat & 3])
    order = np.lexsort(key[::-1])
    assert np.array_equal(order, np.arange(len(h)))
    d = np.diff(key, axis=1)
    first_diff = np.where(d != 0, 1, 0).argmax(axis=0)
    assert (d[first_diff, np.arange(d.shape[1])] > 0).all() if len(h) > 1 else True
    # inside their records, within the pair's mismatch budget
    assert (h["pos"].astype(np.int64) + L <= lengths[h["record"]]).all()
    assert (h["mism"] <= np.asarray(wl.k)[pair]).all()
    # amplicons: geometry from their two sites, orientation from their strands and primers
    hi_, hj = h[a["hit_i"]], h[a["hit_j"]]
    pi, pj = hi_["pattern"].astype(np.int64), hj["pattern"].astype(np.int64)
    assert (hi_["record"] == a["record"]).all() and (hj["record"] == a["record"]).all()
    assert ((pi >> 2) == a["pair"]).all() and ((pj >> 2) == a["pair"]).all()
    assert (((pi >> 1) & 1) == 0).all() and (((pj >> 1) & 1) == 1).all()   # + anchor, - partner
    assert (a["start"] == hi_["pos"]).all()
    assert (a["end"].astype(np.int64) == hj["pos"].astype(np.int64) + plen[pj >> 2, pj & 1]).all()
    length = a["end"].astype(np.int64) - a["start"].astype(np.int64)
    assert ((length >= wl.min_len) & (length <= wl.max_len)).all()
    expect_orient = np.select([(pi & 1) == 0, True], [np.where((pj & 1) == 1, 0, 2), np.where((pj & 1) == 0, 1, 3)])
    assert (a["orient"] == expect_orient).all()
    assert ((1 << a["orient"].astype(np.int64)) & wl.orient_mask).all()
    if out.field_off is None:
        return
    # every extracted field has the length the trimming and clipping rules give
    off = out.field_off
    flen = np.diff(off).reshape(-1)[: 5 * len(a)].reshape(len(a), 5) if len(a) else np.zeros((0, 5), np.int64)
    s_i, e_j = a["start"].astype(np.int64), a["end"].astype(np.int64)
    e_i = s_i + plen[pi >> 2, pi & 1]
    s_j = hj["pos"].astype(np.int64)
    want0 = np.maximum(0, s_j - e_i) if wl.trim else e_j - s_i
    assert np.array_equal(flen[:, 0], want0)
    rec_len = lengths[a["record"]]
    rc = a["orient"] == 1
    fb = np.where(rc, np.minimum(e_j + wl.fb_len, rec_len) - e_j, s_i - np.maximum(0, s_i - wl.fb_len))
    rb = np.where(rc, s_i - np.maximum(0, s_i - wl.rb_len), np.minimum(e_j + wl.rb_len, rec_len) - e_j)
    assert np.array_equal(flen[:, 1], fb) and np.array_equal(flen[:, 2], rb)
    assert np.array_equal(flen[:, 3], e_i - s_i) and np.array_equal(flen[:, 4], e_j - s_j)


def _sample(n_records, count, seed):
    st = synth.Stream(synth.make_key(seed, 4242, 0))
    out = set()
    while len(out) < min(count, n_records):
        out.add(st.randint(0, n_records - 1))
    return sorted(out)


def test_plain_scale_full(engine):
    """2,000 genomes (7.54 Gbp), one pair, k=3, trimming and 16-nt barcodes: 12 sampled genomes
    against the oracle (sites, amplicons, Tm, sequences), invariants over everything."""
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl = synth.plain_scale()
    p = Params.from_workload(wl)
    batch = engine.pack(wl.seq, wl.offsets, wl.genome_ids)
    try:
        out, info = _plan_output(engine, batch, p)
    finally:
        ah.ah_batch_free(batch)
    assert info["n_hits"] == len(out.hits) and len(out.amps) > 2000
    _check_properties(out, wl, wl.lengths().astype(np.int64))
    recs = _sample(wl.n_records, 12, 1)
    ref = oracle.run(wl.subset(recs))
    sub = compare.Restricted(out, recs)
    compare.assert_same_hits(sub, ref)
    compare.assert_same_amplicons(sub, ref, filtered=False)
    compare.assert_same_sequences(sub, ref)


def test_dense_full(engine):
    """5,000 genomes (17.5 Gbp) with tandem repeats and 18-nt primers with 9 degenerate codes, k=4,
    annotated without sequences as the bench runs it: sites and amplicons of 4 sampled genomes
    against the oracle, Tm of 6 sampled amplicons (the oracle enumerates every variant of both
    primers), invariants over everything."""
    import torch

    import synth.gpu as sg
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl = sg.dense()
    recs = _sample(wl.n_records, 4, 2)
    host = wl.host_subset(recs)
    p = Params.from_workload(wl)
    batch = engine.pack_device(wl.d_seq.data_ptr(), wl.offsets.astype(np.uint64), wl.genome_ids)
    ah.ah_ctx_synchronize(engine.ctx)
    wl.d_seq = None
    torch.cuda.empty_cache()
    try:
        out, info = _plan_output(engine, batch, p, with_seqs=wl.extract)
    finally:
        ah.ah_batch_free(batch)
    lengths = np.diff(wl.offsets).astype(np.int64)
    assert len(out.hits) > wl.total_bp // 1000 and len(out.amps) > wl.total_bp // 2000   # ~2 sites, ~1 amplicon per kb
    _check_properties(out, wl, lengths)
    sub = compare.Restricted(out, recs)
    ref_hits = oracle.scan(host)
    assert compare.gpu_hit_tuples(sub.hits) == compare.oracle_hit_tuples(ref_hits)
    ref_amps = oracle.pair(host, ref_hits)
    assert sorted(compare.gpu_amp_keys(sub)) == sorted(compare.oracle_amp_keys(ref_hits, ref_amps))
    # Tm (reading R13, R14) and sequences of a few amplicons
    st = synth.Stream(synth.make_key(3, 4243, 0))
    picks = sorted({st.randint(0, len(sub.amps) - 1) for _ in range(6)}) if len(sub.amps) else []
    comp = {"A": "T", "C": "G", "G": "C", "T": "A"}
    for m in picks:
        a = sub.amps[m]
        g = host.seq[host.offsets[a["record"]]:host.offsets[a["record"] + 1]].tobytes().decode().upper()
        tms = []
        for hidx in (a["hit_i"], a["hit_j"]):
            x = sub.hits[hidx]
            pat = int(x["pattern"])
            primer = (wl.fwd if (pat & 1) == 0 else wl.rev)[pat >> 2]
            site = g[int(x["pos"]):int(x["pos"]) + len(primer)]
            if (pat >> 1) & 1:
                site = "".join(comp[c] for c in reversed(site))
            tms.append(oracle.tm_site(primer, site, wl.tm))
        if any(t is None for t in tms):
            assert a["flags"] & 4
        else:
            assert abs(float(a["tm"]) - min(tms)) <= compare.TM_TOL


def test_batched_full(engine):
    """50,000 genomes (84.5 Gbp) and 8 pairs in one plan: 16 sampled genomes against the oracle
    (sites, amplicons, Tm, sequences), invariants over everything."""
    import torch

    import synth.gpu as sg
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl = sg.batched()
    recs = _sample(wl.n_records, 16, 3)
    host = wl.host_subset(recs)
    p = Params.from_workload(wl)
    batch = engine.pack_device(wl.d_seq.data_ptr(), wl.offsets.astype(np.uint64), wl.genome_ids)
    ah.ah_ctx_synchronize(engine.ctx)
    wl.d_seq = None
    torch.cuda.empty_cache()
    try:
        out, info = _plan_output(engine, batch, p)
    finally:
        ah.ah_batch_free(batch)
    _check_properties(out, wl, np.diff(wl.offsets).astype(np.int64))
    ref = oracle.run(host)
    sub = compare.Restricted(out, recs)
    compare.assert_same_hits(sub, ref)
    compare.assert_same_amplicons(sub, ref, filtered=False)
    compare.assert_same_sequences(sub, ref)


def test_serving_full():
    """The serving database at full size (40,000 genomes, 151.5 Gbp resident, drawn and packed in
    ranges as the bench does), 8 slots, the first requests of the Poisson trace with at most 12
    pairs submitted together: each result, restricted to two sampled records of its range, equals
    the oracle on those records (sites, amplicons, Tm, sequences)."""
    import torch

    import synth.gpu as sg
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Engine, Output

    n_db = 40_000
    lengths, _ = sg.serving_layout(n_genomes=n_db)
    trace = [r for r in synth.serving_trace(synth.SEED, 60, 200.0, n_db) if len(r["fwd"]) <= 12][:6]
    st = synth.Stream(synth.make_key(7, 4244, 0))
    picks = {i: sorted({r["first_record"] + st.randint(0, r["n_records"] - 1) for _ in range(2)})
             for i, r in enumerate(trace)}
    wanted = sorted({g for v in picks.values() for g in v})
    host = {}
    eng = Engine(0)
    db = ah.ah_batch_create(eng.ctx, np.asarray(lengths, dtype=np.uint64))
    try:
        for first, d, offs in sg.serving_db_chunks(n_genomes=n_db):
            for g in wanted:
                if first <= g < first + len(offs) - 1:
                    host[g] = d[int(offs[g - first]):int(offs[g - first + 1])].cpu().numpy().copy()
            ah.ah_batch_pack_range(eng.ctx, db, first, d.data_ptr(), offs.astype(np.uint64))
            del d
            torch.cuda.empty_cache()
        srv = ah.ah_server_create(db, n_slots=8)
        try:
            keys = ("fwd", "rev", "k", "clamp", "first_record", "n_records", "min_len", "max_len", "orient_mask")
            tickets = [ah.ah_server_submit(srv, **{k: r[k] for k in keys}) for r in trace]
            results = [ah.ah_server_wait(srv, t) for t in tickets]
        finally:
            ah.ah_server_destroy(srv)
    finally:
        ah.ah_batch_free(db)
        eng.close()
    for i, (r, got) in enumerate(zip(trace, results)):
        recs = picks[i]
        seq = np.concatenate([host[g] for g in recs])
        offs = np.concatenate([[0], np.cumsum([len(host[g]) for g in recs])]).astype(np.int64)
        wl = synth.Workload("serving-sample", seq, offs, np.asarray(recs, dtype=np.uint32), list(r["fwd"]),
                            list(r["rev"]), list(r["k"]), r["clamp"], r["min_len"], r["max_len"], r["orient_mask"],
                            synth.TmParams(min_tm=None), False, 0, 0)
        ref = oracle.run(wl)
        sub = compare.Restricted(Output(got["hits"], got["amps"], got["arena"], got["field_off"]), recs)
        compare.assert_same_hits(sub, ref)
        compare.assert_same_amplicons(sub, ref, filtered=False)
        compare.assert_same_sequences(sub, ref)
