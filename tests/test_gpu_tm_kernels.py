"""The two degenerate-site Tm kernels against the oracle, through the C ABI (needs a GPU).

The kernel generated per primer set (straight-line chains, terms regrouped onto the degenerate
positions) and the kernel built into the library must both give the oracle's maximum over every
concrete variant (Section "Primer degeneracy") within 1e-9 degC, on primer shapes chosen to reach
every case of the generated chain: degenerate runs at the duplex's ends (terminal-mismatch steps
stored per site), adjacent degenerate positions inside (steps read in place), degenerate positions
two apart and further (terms split between their neighbours), three-choice codes, concrete
primers, the shortest and longest primers.
"""
import time

import numpy as np
import pytest

import oracle
import synth
from tests import compare

pytestmark = pytest.mark.gpu

# (forward, reverse, mismatch budget): each pair is planted with substitutions, 4 sites per record
SHAPES = [
    ("NNRYTGACCGTAGSAN", "NAGYCGATWKSGNACT", 3),   # degenerate runs at both ends
    ("BDTGACCGHVAGTCAN", "VHGYCGATWASGTACB", 3),   # three-choice codes at the ends and inside
    ("RAYASAKAMAWAGTCC", "TGYARAYCAGATCACG", 2),   # degenerate positions two apart
    ("ACGTTGCAGGTACCAT", "TTGGCCAAGCTAGCTA", 2),   # concrete primers: one variant each
    ("GACNTGAGCTAC", "TCAGGRTTCMAG", 1),           # one degenerate position each
    ("ACGTRYKMACGTSWBDACGTHVGGACGTACGT", "TGCAACGTAGCTAGCTNNAGCTAGGCATGCAA", 2),  # 32 nt
    ("SRNNAWCRWYAAGTSACC", "ATCWKSRANTMRRNATAA", 3),  # the dense workload's shape
]
# salt method, Na (mM), Mg (mM), selfcomp: one per shape, round robin
SALTS = [(5, 50.0, 0.0, 0), (4, 10.0, 0.0, 0), (1, 50.0, 1.5, 0), (0, 50.0, 0.0, 1), (3, 200.0, 0.0, 0),
         (2, 50.0, 0.0, 0), (5, 20.0, 2.0, 1)]


@pytest.fixture(scope="module")
def engine():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2511_00170_gb300.pipeline import Engine

    e = Engine(0)
    yield e
    e.close()


def _planted_case(i: int, fwd: str, rev: str, k: int):
    wl = synth.random_small(900 + i, n_records=6, len_lo=3000, len_hi=8000, n_pairs=1, plant=0, clamp=3,
                            min_len=20, max_len=3000, fb=0, rb=0, trim=False)
    wl.fwd, wl.rev, wl.k = [fwd], [rev], [k]
    st = synth.Stream(synth.make_key(900 + i, 31, 7))
    wl.planted = []
    for g in range(wl.n_records):
        synth._plant(wl.seq, wl.offsets, g, st, 4, fwd, rev, 0, lambda s: s.randint(20, 400), k, wl.planted)
    method, na, mg, selfcomp = SALTS[i % len(SALTS)]
    wl.tm.saltcorr, wl.tm.Na, wl.tm.Mg, wl.tm.selfcomp = method, na, mg, selfcomp
    wl.tm.min_tm = None
    return wl


def _step(engine, wl, mode):
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    ah.ah_ctx_set_tm_kernel(engine.ctx, mode)
    ah.ah_ctx_stats_reset(engine.ctx)
    batch = engine.pack(wl.seq, wl.offsets, wl.genome_ids)
    try:
        out = engine.step(batch, Params.from_workload(wl), with_seqs=False)
    finally:
        ah.ah_batch_free(batch)
        st = ah.ah_ctx_stats_get(engine.ctx)
        ah.ah_ctx_set_tm_kernel(engine.ctx, 0)
    return out, st


@pytest.mark.parametrize("i", range(len(SHAPES)))
def test_generated_and_builtin_match_oracle(engine, i):
    from paper_2511_00170_gb300 import ah

    fwd, rev, k = SHAPES[i]
    st, log = ah.ah_tm_kernel_check([fwd, rev])
    assert st == 0, log
    wl = _planted_case(i, fwd, rev, k)
    ref = oracle.run(wl, with_seqs=False)
    assert len(ref.amps) > 0, "the planted sites form no amplicon"
    gen, s_gen = _step(engine, wl, 0)
    assert s_gen["tm_generated"] == 1 and s_gen["tm_builtin"] == 0, s_gen
    bui, s_bui = _step(engine, wl, 1)
    assert s_bui["tm_builtin"] == 1 and s_bui["tm_generated"] == 0, s_bui
    for out in (gen, bui):
        compare.assert_same_hits(out, ref)
        compare.assert_same_amplicons(out, ref, filtered=False)
    # the two kernels: the same amplicons in the same order, Tm within the tolerance
    assert np.array_equal(gen.amps[["hit_i", "hit_j", "flags"]], bui.amps[["hit_i", "hit_j", "flags"]])
    a, b = gen.amps["tm"], bui.amps["tm"]
    both = ~np.isnan(a)
    assert np.array_equal(both, ~np.isnan(b))
    assert np.all(np.abs(a[both] - b[both]) <= compare.TM_TOL)


def test_background_compile(engine):
    """Mode 2 takes the built-in kernel while the primer set's kernel compiles on a host thread, then
    the generated one; both results match the oracle."""
    fwd, rev = "GTRCAGYTAGGCAMCT", "ACKTGGACRTGCAYAG"   # used by no other test: compiled here first
    wl = _planted_case(50, fwd, rev, 2)
    ref = oracle.run(wl, with_seqs=False)
    first, s1 = _step(engine, wl, 2)
    assert s1["tm_builtin"] == 1 and s1["tm_generated"] == 0, s1
    compare.assert_same_amplicons(first, ref, filtered=False)
    deadline = time.time() + 120.0
    while True:
        later, s2 = _step(engine, wl, 2)
        if s2["tm_generated"] == 1:
            break
        assert time.time() < deadline, "the generated Tm kernel never became ready"
        time.sleep(0.5)
    compare.assert_same_amplicons(later, ref, filtered=False)


def test_large_sets_take_the_builtin_kernel(engine):
    """Primers whose adjacent degenerate runs exceed the compile budget stay on the built-in kernel."""
    fwd, rev = "NNNNNNNNACGTACGA", "TGCATGCATTGCAGCA"   # 7 adjacent N steps: 112 transitions
    wl = _planted_case(60, fwd, rev, 1)
    ref = oracle.run(wl, with_seqs=False)
    out, st = _step(engine, wl, 0)
    assert st["tm_builtin"] == 1 and st["tm_generated"] == 0, st
    compare.assert_same_amplicons(out, ref, filtered=False)


def test_per_primer_launches(engine):
    """The generated kernel launched once per primer (as it runs for many sites) gives every site the
    Tm of a single launch, bit for bit, and the oracle's."""
    from paper_2511_00170_gb300 import ah

    fwd, rev, k = SHAPES[6]
    wl = _planted_case(70, fwd, rev, k)
    ref = oracle.run(wl, with_seqs=False)
    runs = []
    for sites in (1, 2**64 - 1):
        ah.ah_ctx_set_tm_split(engine.ctx, sites)
        try:
            runs.append(_step(engine, wl, 0))
        finally:
            ah.ah_ctx_set_tm_split(engine.ctx, 0)
    (split, s_split), (one, s_one) = runs
    assert s_split["tm_generated"] == 1 and s_one["tm_generated"] == 1
    assert s_split["kernel_launches"] == s_one["kernel_launches"] + 1   # two primers: two launches
    compare.assert_same_amplicons(split, ref, filtered=False)
    assert np.array_equal(split.amps["tm"].view(np.int64), one.amps["tm"].view(np.int64))
