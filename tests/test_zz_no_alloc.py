"""The allocation-free pairing entry point, through the C ABI (needs a GPU; collected last).

Some callers of this library cannot allocate device memory while they run a step. Their
application may already own all GPU memory through its own pool, or they may be unable to accept
the synchronisation a cudaMalloc brings. ah_pair_amplicons_noalloc serves them: it pairs sites
into amplicons using only buffers the caller passes in, plus one fixed scratch array inside the
library. Here the test plays that caller. It owns the output buffer and the primer-length table,
hands their device addresses to the entry point, and checks the records byte for byte against the
allocating entry point ah_pair_amplicons, on two different workloads called back to back.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2511_00170_gb300.pipeline import Engine

    e = Engine(0)
    yield e
    e.close()


def _sites_and_reference(engine, wl):
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    p = Params.from_workload(wl)
    pr = engine.primers(p)
    batch = engine.pack(wl.seq, wl.offsets)
    hits = ah.ah_scan_primers(engine.ctx, batch, pr)
    amps = ah.ah_pair_amplicons(engine.ctx, batch, pr, hits, p.min_len, p.max_len, p.orient_mask)
    ref = ah.ah_amplicons_copy(amps)
    ah.ah_amplicons_free(amps)
    return p, batch, hits, ref


def _pattern_lengths(p):
    lens = []
    for f, r in zip(p.fwd, p.rev):
        lens += [len(f), len(r), len(f), len(r)]   # orient = 2 * strand + primer
    return lens


def _noalloc(engine, p, hits, capacity):
    import torch

    from paper_2511_00170_gb300 import ah

    d_hits, d_off = ah.ah_hits_device(hits)
    n_hits = ah.ah_hits_count(hits)
    plen = torch.tensor(_pattern_lengths(p), dtype=torch.uint8, device="cuda")
    out = torch.empty(max(1, capacity) * ah.AMP_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    ah.ah_ctx_synchronize(engine.ctx)
    torch.cuda.synchronize()
    n = ah.ah_pair_amplicons_noalloc(ah.ah_ctx_stream(engine.ctx), d_hits, n_hits, d_off, plen.data_ptr(), p.min_len,
                                     p.max_len, p.orient_mask, out.data_ptr(), capacity)
    ah.ah_ctx_synchronize(engine.ctx)
    return out[:n * ah.AMP_DTYPE.itemsize].cpu().numpy().view(ah.AMP_DTYPE)


def test_noalloc_pairing_matches_allocating_entry_point(engine):
    from paper_2511_00170_gb300 import ah

    workloads = [synth.plain_small(n_genomes=6, len_lo=100_000, len_hi=300_000),
                 synth.batched(n_genomes=30, len_lo=2e3, len_hi=2e5, n_pairs=4)]
    for wl in workloads:   # two calls in a row; the second sees the first call's scratch contents
        p, batch, hits, ref = _sites_and_reference(engine, wl)
        try:
            assert len(ref) > 0
            got = _noalloc(engine, p, hits, len(ref) + 7)
            assert len(got) == len(ref)
            assert got.tobytes() == ref.tobytes()
        finally:
            ah.ah_hits_free(hits)
            ah.ah_batch_free(batch)


def test_noalloc_pairing_reports_limits(engine):
    from paper_2511_00170_gb300 import ah

    wl = synth.plain_small(n_genomes=4, len_lo=100_000, len_hi=200_000)
    p, batch, hits, ref = _sites_and_reference(engine, wl)
    try:
        assert len(ref) > 1
        with pytest.raises(ah.AhError) as e:
            _noalloc(engine, p, hits, len(ref) - 1)
        assert e.value.status == ah.AH_EOVERFLOW
        with pytest.raises(ah.AhError) as e:
            ah.ah_pair_amplicons_noalloc(0, 1, ah.AH_PAIR_NOALLOC_MAX_SITES + 1, 1, 1, 50, 2000, 15, 1, 1)
        assert e.value.status == ah.AH_EINVAL
        # the failed calls leave the entry point usable
        got = _noalloc(engine, p, hits, len(ref))
        assert got.tobytes() == ref.tobytes()
    finally:
        ah.ah_hits_free(hits)
        ah.ah_batch_free(batch)
