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


def _periodic(periods, tail):
    """One record of (30 A, 30 T) periods and a final run of `tail` A: with the all-A primers below
    and k = 0 every period holds exactly 80 sites (F+ 21, R+ 19, F- 21, R- 19) and 40 amplicons (the
    last + site of each A run pairs with every - site of the next T run), and the tail 2 * tail - 20
    sites and no amplicon.  Partner counts are spread over every block of the prefix sums."""
    g = ("A" * 30 + "T" * 30) * periods + "A" * tail
    wl = synth.random_small(2, n_records=1, len_lo=10, len_hi=10, n_pairs=1, plant=0)
    wl.seq = np.frombuffer(g.encode(), dtype=np.uint8).copy()
    wl.offsets = np.array([0, len(g)], dtype=np.int64)
    wl.genome_ids = np.zeros(1, dtype=np.uint32)
    wl.fwd, wl.rev, wl.k, wl.clamp = ["A" * 10], ["A" * 12], [0], 2
    wl.min_len, wl.max_len, wl.orient_mask = 20, 200, 15
    return wl


@pytest.mark.parametrize("periods,tail", [(12_500, 0), (13_107, 18)])
def test_noalloc_pairing_many_blocks(engine, periods, tail):
    """About a million sites (489 blocks of partial sums) and exactly AH_PAIR_NOALLOC_MAX_SITES
    (all 512), so that the carry between blocks of the prefix sums is exercised."""
    from paper_2511_00170_gb300 import ah

    wl = _periodic(periods, tail)
    p, batch, hits, ref = _sites_and_reference(engine, wl)
    try:
        n_hits = ah.ah_hits_count(hits)
        assert n_hits == 80 * periods + (2 * tail - 20 if tail else 0)
        assert n_hits > 2 * 2048
        if tail:
            assert n_hits == ah.AH_PAIR_NOALLOC_MAX_SITES
        assert len(ref) == 40 * periods
        for _ in range(2):   # two calls in a row over the same shared scratch
            got = _noalloc(engine, p, hits, len(ref))
            assert len(got) == len(ref)
            assert got.tobytes() == ref.tobytes()
    finally:
        ah.ah_hits_free(hits)
        ah.ah_batch_free(batch)


_FIRST_CALL = r'''
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
import oracle
import synth
from paper_2511_00170_gb300 import ah

wl = synth.plain_small(n_genomes=3, len_lo=100_000, len_hi=200_000)
o = oracle.scan(wl)
orient = 2 * o["strand"].astype(np.int64) + o["primer"]
order = np.lexsort((orient, o["pos"], o["record"], o["pair"]))   # the library's site order
hits = np.zeros(len(o), dtype=ah.HIT_DTYPE)
hits["record"], hits["pos"], hits["mism"] = o["record"][order], o["pos"][order], o["mism"][order]
hits["pattern"] = 4 * o["pair"][order].astype(np.int64) + orient[order]
n_pairs = len(wl.fwd)
pair_off = np.searchsorted(o["pair"][order], np.arange(n_pairs + 1)).astype(np.uint64)
plen = []
for f, r in zip(wl.fwd, wl.rev):
    plen += [len(f), len(r), len(f), len(r)]
d_hits = torch.from_numpy(hits.view(np.uint8).copy()).cuda()
d_off = torch.from_numpy(pair_off.view(np.uint8).copy()).cuda()
d_plen = torch.tensor(plen, dtype=torch.uint8, device="cuda")
cap = 4096
d_out = torch.empty(cap * ah.AMP_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
torch.cuda.synchronize()
# the first call of the library in this process
n = ah.ah_pair_amplicons_noalloc(0, d_hits.data_ptr(), len(hits), d_off.data_ptr(), d_plen.data_ptr(), wl.min_len,
                                 wl.max_len, wl.orient_mask, d_out.data_ptr(), cap)
torch.cuda.synchronize()
got = d_out[:n * ah.AMP_DTYPE.itemsize].cpu().numpy().view(ah.AMP_DTYPE)

from paper_2511_00170_gb300.pipeline import Engine, Params
e = Engine(0)
p = Params.from_workload(wl)
batch = e.pack(wl.seq, wl.offsets)
h = ah.ah_scan_primers(e.ctx, batch, e.primers(p))
assert ah.ah_hits_copy(h).tobytes() == hits.tobytes(), "oracle sites differ from the scan's"
a = ah.ah_pair_amplicons(e.ctx, batch, e.primers(p), h, p.min_len, p.max_len, p.orient_mask)
ref = ah.ah_amplicons_copy(a)
assert n > 0 and len(got) == len(ref), (n, len(ref))
assert got.tobytes() == ref.tobytes()
print("first-call ok", n)
'''


def test_noalloc_pairing_as_first_call_of_a_process(engine):
    """In a fresh process whose first library call is the allocation-free pairing (its device code and
    scratch array are set up by that call), the result equals the allocating entry point's.  (The
    engine fixture only makes sure the library is built; it lives in this test process.)"""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "first-call ok" in r.stdout
