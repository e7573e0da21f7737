"""Batched forms through the C ABI (needs a GPU): the graph-captured plan (autotuned, persistent or
not, with capacities that overflow and grow) and the one-launch-per-record-per-pair scan give
exactly the outputs of the regular path, which the parity tests pin to the oracle."""
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


def _same(a, b):
    assert a.hits.tobytes() == b.hits.tobytes()
    assert a.amps.tobytes() == b.amps.tobytes()
    assert (a.arena or b"") == (b.arena or b"")
    if a.field_off is not None:
        assert np.array_equal(a.field_off, b.field_off)


@pytest.mark.parametrize("persistent,autotune,queue", [(0, False, 0), (1, False, 0), (-1, True, 0), (0, False, 1),
                                                       (1, False, 1)])
def test_plan_matches_regular_path_and_oracle(engine, persistent, autotune, queue):
    """The plan (one CTA per tile or persistent CTAs, candidates emitted where found or queued per
    warp) gives the regular path's bytes and the oracle's sites, amplicons and sequences."""
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl = synth.batched(n_genomes=60, len_lo=5e3, len_hi=4e5, n_pairs=4)
    wl.tm.min_tm = 30.0
    wl.trim, wl.fb_len, wl.rb_len = True, 12, 9
    p = Params.from_workload(wl)
    batch = engine.pack(wl.seq, wl.offsets)
    ah.ah_ctx_set_scan_circuit(engine.ctx, 0, 1024, queue)
    try:
        ref = engine.step(batch, p)
        plan = engine.plan(batch, p, with_seqs=True, autotune=autotune, persistent=persistent)
        try:
            for _ in range(3):   # replays of the same graph
                ah.ah_plan_run(plan, engine.ctx)
            out = engine.plan_output(plan)
            info = ah.ah_plan_info_get(plan)
        finally:
            ah.ah_plan_free(plan)
    finally:
        ah.ah_batch_free(batch)
        ah.ah_ctx_set_scan_circuit(engine.ctx, 0, 1024, 0)
    _same(out, ref)
    assert info["n_hits"] == len(ref.hits) and info["n_kept"] == len(ref.amps)
    if persistent == 1:
        assert info["persistent"] == 1
    if not autotune:
        assert info["emit_queue"] == queue
    orc = oracle.run(wl)
    compare.assert_same_hits(out, orc)
    compare.assert_same_amplicons(out, orc, filtered=True)
    compare.assert_same_sequences(out, orc)


def test_plan_grows_capacities(engine):
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl = synth.plain_small(n_genomes=5, len_lo=100_000, len_hi=300_000)
    p = Params.from_workload(wl)
    batch = engine.pack(wl.seq, wl.offsets)
    try:
        ref = engine.step(batch, p)
        ah.ah_ctx_set_scan_config(engine.ctx, 128, 8, 16, 0)
        plan = engine.plan(batch, p, hit_capacity=3, amp_capacity=1, arena_capacity=5)
        try:
            with pytest.raises(ah.AhError) as e:
                ah.ah_plan_launch(plan, engine.ctx)
                ah.ah_plan_check(plan, engine.ctx)
            assert e.value.status == ah.AH_EOVERFLOW
            ah.ah_plan_run(plan, engine.ctx)
            out = engine.plan_output(plan)
        finally:
            ah.ah_plan_free(plan)
            ah.ah_ctx_set_scan_config(engine.ctx, 128, 8, 256, 0)
    finally:
        ah.ah_batch_free(batch)
    _same(out, ref)


def test_per_record_scan_matches(engine):
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl = synth.batched(n_genomes=25, len_lo=1e3, len_hi=3e5, n_pairs=3)
    p = Params.from_workload(wl)
    batch = engine.pack(wl.seq, wl.offsets)
    try:
        pr = engine.primers(p)
        h1 = ah.ah_scan_primers(engine.ctx, batch, pr)
        h2 = ah.ah_scan_primers_per_record(engine.ctx, batch, pr)
        a, b = ah.ah_hits_copy(h1), ah.ah_hits_copy(h2)
        ah.ah_hits_free(h1)
        ah.ah_hits_free(h2)
    finally:
        ah.ah_batch_free(batch)
    assert len(a) > 0 and a.tobytes() == b.tobytes()


def test_plan_replays_are_timed_and_counted(engine):
    """With timing on, each replay's scan node is timed by its own event pair (more replays than the
    ring of timed graphs holds, so slots are reused after their timings are read) and every kernel
    node of the graph is counted; untimed replays afterwards leave the counters alone."""
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl = synth.batched(n_genomes=20, len_lo=5e3, len_hi=2e5, n_pairs=2)
    p = Params.from_workload(wl)
    batch = engine.pack(wl.seq, wl.offsets)
    try:
        plan = engine.plan(batch, p, with_seqs=True)
        try:
            ah.ah_plan_run(plan, engine.ctx)
            ah.ah_ctx_stats_reset(engine.ctx)
            ah.ah_ctx_set_timing(engine.ctx, True)
            n = 21
            for _ in range(n):
                ah.ah_plan_launch(plan, engine.ctx)
            ah.ah_ctx_set_timing(engine.ctx, False)
            st = ah.ah_ctx_stats_get(engine.ctx)
            assert st["scan_launches"] == n and st["scan_bases"] == n * int(wl.total_bp)
            assert st["scan_ms"] > 0
            per_replay = st["kernel_launches"] // n
            assert st["kernel_launches"] == n * per_replay and per_replay >= 10
            for _ in range(2):
                ah.ah_plan_launch(plan, engine.ctx)
            ah.ah_ctx_synchronize(engine.ctx)
            st2 = ah.ah_ctx_stats_get(engine.ctx)
            assert st2["scan_launches"] == n and st2["scan_ms"] == st["scan_ms"]
            assert st2["kernel_launches"] == (n + 2) * per_replay
            ah.ah_plan_check(plan, engine.ctx)
        finally:
            ah.ah_plan_free(plan)
    finally:
        ah.ah_batch_free(batch)


def test_plan_copy_results(engine):
    """The direct copy of a run's results into caller buffers equals the results objects, and buffers
    that are too small are refused with AH_EOVERFLOW."""
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl = synth.batched(n_genomes=20, len_lo=5e3, len_hi=2e5, n_pairs=3)
    wl.trim, wl.fb_len, wl.rb_len = True, 10, 7
    p = Params.from_workload(wl)
    batch = engine.pack(wl.seq, wl.offsets)
    try:
        plan = engine.plan(batch, p, with_seqs=True)
        try:
            ah.ah_plan_run(plan, engine.ctx)
            ref = engine.plan_output(plan)
            i = ah.ah_plan_info_get(plan)
            hits = np.zeros(i["n_hits"] + 3, ah.HIT_DTYPE)
            amps = np.zeros(i["n_kept"] + 3, ah.AMP_DTYPE)
            arena = np.zeros(i["arena_bytes"] + 3, np.uint8)
            fo = np.zeros(5 * i["n_kept"] + 1, np.uint64)
            ah.ah_plan_copy_results(plan, engine.ctx, hits, amps, arena, fo)
            assert hits[:i["n_hits"]].tobytes() == ref.hits.tobytes()
            assert amps[:i["n_kept"]].tobytes() == ref.amps.tobytes()
            assert arena[:i["arena_bytes"]].tobytes() == (ref.arena or b"")
            assert np.array_equal(fo, ref.field_off)
            with pytest.raises(ah.AhError) as e:
                ah.ah_plan_copy_results(plan, engine.ctx, hits[:max(0, i["n_hits"] - 1)], None, None, None)
            assert e.value.status == ah.AH_EOVERFLOW or i["n_hits"] == 0
        finally:
            ah.ah_plan_free(plan)
    finally:
        ah.ah_batch_free(batch)


@pytest.mark.parametrize("persistent", [0, 1])
def test_launch_host_matches_launch(engine, persistent):
    """The step on genomes in host memory, each range of scan tiles launched as its bases land
    (ah_plan_launch_host), equals the plan's replay on the same genomes packed beforehand.  The
    genomes span two staged chunks of the upload, and the plan's batch holds other bases before
    the call, so a range scanned before its bases landed would show."""
    import torch

    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl = synth.batched(n_genomes=200, n_pairs=2)
    assert wl.total_bp > (256 << 20)
    wl.trim, wl.fb_len, wl.rb_len = True, 10, 8
    p = Params.from_workload(wl)
    text = torch.empty(wl.total_bp, dtype=torch.uint8, pin_memory=True)
    text.numpy()[:] = wl.seq
    other = torch.full((wl.total_bp,), ord("A"), dtype=torch.uint8, pin_memory=True)
    offs = np.ascontiguousarray(wl.offsets, dtype=np.uint64)
    batch = engine.pack(wl.seq, wl.offsets)
    try:
        plan = engine.plan(batch, p, with_seqs=True, persistent=persistent)
        try:
            ah.ah_plan_run(plan, engine.ctx)
            ref = engine.plan_output(plan)
            assert len(ref.amps) > 0
            for _ in range(2):
                ah.ah_batch_pack_range(engine.ctx, batch, 0, other.data_ptr(), offs)
                ah.ah_plan_launch_host(plan, text.data_ptr(), offs, engine.ctx)
                ah.ah_plan_check(plan, engine.ctx)
                _same(engine.plan_output(plan), ref)
        finally:
            ah.ah_plan_free(plan)
    finally:
        ah.ah_batch_free(batch)


@pytest.mark.parametrize("persistent", [0, 1])
def test_launch_packed_matches_launch(engine, persistent):
    """The step on 2-bit batches in host memory, each range of scan tiles launched as its planes land
    (ah_plan_launch_packed), equals the plan's replay on the batch packed from text.  The planes span
    several copy chunks, the genomes carry runs of invalid bases (sparse invalid words), and the plan's
    batch holds other bases before the call, so a range scanned early, or an invalid word not yet
    written, would show."""
    import torch

    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl = synth.batched(n_genomes=800, n_pairs=2)
    assert wl.total_bp > (2 * 256 << 20)
    wl.trim, wl.fb_len, wl.rb_len = True, 10, 8
    p = Params.from_workload(wl)
    other = torch.full((wl.total_bp,), ord("C"), dtype=torch.uint8, pin_memory=True)
    offs = np.ascontiguousarray(wl.offsets, dtype=np.uint64)
    batch = engine.pack(wl.seq, wl.offsets)
    try:
        v = ah.ah_batch_view_get(batch)
        pl_t = torch.empty(v["n_groups"] * 8, dtype=torch.uint8, pin_memory=True)
        planes = pl_t.numpy().view(np.uint32).reshape(-1, 2)
        _, groups, words = ah.ah_batch_export(batch, planes)
        assert len(groups) > 0
        plan = engine.plan(batch, p, with_seqs=True, persistent=persistent)
        try:
            ah.ah_plan_run(plan, engine.ctx)
            ref = engine.plan_output(plan)
            assert len(ref.amps) > 0
            for _ in range(2):
                ah.ah_batch_pack_range(engine.ctx, batch, 0, other.data_ptr(), offs)
                ah.ah_plan_launch_packed(plan, planes, groups, words, engine.ctx)
                ah.ah_plan_check(plan, engine.ctx)
                _same(engine.plan_output(plan), ref)
            # a group past the batch is refused before anything is enqueued
            bad = np.array([v["n_groups"]], dtype=np.uint64)
            with pytest.raises(ah.AhError) as e:
                ah.ah_plan_launch_packed(plan, planes, bad, np.array([1], dtype=np.uint32), engine.ctx)
            assert e.value.status == ah.AH_EINVAL
        finally:
            ah.ah_plan_free(plan)
    finally:
        ah.ah_batch_free(batch)


def _fasta_text(seq, offsets, width=80):
    """The records as FASTA, `width`-column sequence lines (uint8 array)."""
    parts = []
    for r in range(len(offsets) - 1):
        s = seq[int(offsets[r]):int(offsets[r + 1])]
        L = len(s)
        full = (L // width) * width
        body = np.full(full + full // width, 10, dtype=np.uint8)
        if full:
            body.reshape(-1, width + 1)[:, :width] = s[:full].reshape(-1, width)
        tail = np.concatenate([s[full:], [10]]).astype(np.uint8) if L > full else np.zeros(0, np.uint8)
        parts += [np.frombuffer(b">genome_%d synthetic\n" % r, dtype=np.uint8), body, tail]
    return np.concatenate(parts)


@pytest.mark.parametrize("on_device", [False, True])
def test_launch_fasta_matches_launch(engine, on_device):
    """The step on FASTA text, parsed chunk by chunk as it lands with the completed records packed and
    their tiles scanned at once (ah_plan_launch_fasta), equals the plan's replay on the batch packed
    beforehand; the text spans four copy chunks, and the plan's batch holds other bases before the
    call.  A text missing a record is refused."""
    import torch

    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl = synth.batched(n_genomes=600, n_pairs=2)
    wl.trim, wl.fb_len, wl.rb_len = True, 10, 8
    p = Params.from_workload(wl)
    text = _fasta_text(wl.seq, wl.offsets)
    assert len(text) > 3 * (256 << 20)
    if on_device:
        t_text = torch.from_numpy(text).to("cuda:0")
    else:
        t_text = torch.empty(len(text), dtype=torch.uint8, pin_memory=True)
        t_text.numpy()[:] = text
    other = torch.full((wl.total_bp,), ord("G"), dtype=torch.uint8, pin_memory=True)
    offs = np.ascontiguousarray(wl.offsets, dtype=np.uint64)
    batch = engine.pack(wl.seq, wl.offsets)
    try:
        plan = engine.plan(batch, p, with_seqs=True)
        try:
            ah.ah_plan_run(plan, engine.ctx)
            ref = engine.plan_output(plan)
            assert len(ref.amps) > 0
            for _ in range(2):
                ah.ah_batch_pack_range(engine.ctx, batch, 0, other.data_ptr(), offs)
                ah.ah_plan_launch_fasta(plan, t_text.data_ptr(), len(text), engine.ctx)
                ah.ah_plan_check(plan, engine.ctx)
                _same(engine.plan_output(plan), ref)
            last = int(np.flatnonzero(text == ord(">"))[-1])   # the text without its last record
            with pytest.raises(ah.AhError) as e:
                ah.ah_plan_launch_fasta(plan, t_text.data_ptr(), last, engine.ctx)
            assert e.value.status == ah.AH_EINVAL
            ah.ah_ctx_synchronize(engine.ctx)
        finally:
            ah.ah_plan_free(plan)
    finally:
        ah.ah_batch_free(batch)
