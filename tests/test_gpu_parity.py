"""CUDA path vs oracle, element by element, through the C ABI (needs a GPU).

Hits, amplicons, orientations, trimmed sequences, barcodes and primer snippets must match the
oracle exactly; Tm must agree within 1e-9 C (FP64 on both sides; the tolerance covers summation
order and libm differences, ~1e-13 relative).
"""
import math

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


def _run_both(engine, wl, filtered=True):
    from paper_2511_00170_gb300.pipeline import Params

    ref = oracle.run(wl)
    p = Params.from_workload(wl)
    p_unf = Params.from_workload(wl)
    p_unf.min_tm = None
    batch = engine.pack(wl.seq, wl.offsets, wl.genome_ids)
    try:
        out_unf = engine.step(batch, p_unf, with_seqs=False)
        out = engine.step(batch, p, with_seqs=True)
    finally:
        from paper_2511_00170_gb300 import ah

        ah.ah_batch_free(batch)
    compare.assert_same_hits(out_unf, ref)
    compare.assert_same_hits(out, ref)
    compare.assert_same_amplicons(out_unf, ref, filtered=False)
    compare.assert_same_amplicons(out, ref, filtered=wl.tm.min_tm is not None)
    compare.assert_same_sequences(out, ref)
    return out, ref


def _random_case(seed):
    st = synth.Stream(synth.make_key(seed, 555, 0))
    wl = synth.random_small(seed, n_records=st.randint(1, 6), len_lo=0, len_hi=st.choice([300, 2000, 5000]),
                            n_pairs=st.randint(1, 3), plen_lo=st.randint(4, 12), plen_hi=st.randint(12, 26),
                            n_deg=st.randint(0, 5), k_max=st.randint(0, 4), clamp=st.randint(0, 4),
                            n_frac=st.choice([0.0, 0.01, 0.05]), alphabet=st.choice(["ACGT", "ACGTacgt", "AT", "ACGTTTTT"]),
                            plant=st.randint(0, 4), min_len=st.randint(1, 60), max_len=st.randint(60, 1500),
                            fb=st.randint(0, 20), rb=st.randint(0, 20), trim=bool(st.randint(0, 1)))
    if st.randint(0, 1):
        wl.tm.min_tm = float(st.randint(-20, 40))
    wl.tm.saltcorr = st.choice([5, 5, 5, 0, 1, 2, 3, 4, 6, 7, 7])
    wl.tm.Na = float(st.choice([50, 10, 200]))
    wl.tm.Mg = float(st.choice([0, 0, 1.5, 3]))
    wl.tm.dNTPs = float(st.choice([0, 0.8]))
    return wl


@pytest.mark.parametrize("seed", range(40))
def test_random_small(engine, seed):
    _run_both(engine, _random_case(seed))


def test_plain_small_full(engine):
    """The 16-genome single-pair workload (U(1,3) Mbp, k=2, clamp 3, Tm >= 45 C), every output."""
    out, ref = _run_both(engine, synth.plain_small())
    assert len(ref.hits) > 0 and len(ref.amps) > 0 and ref.keep.any()


def test_edge_records(engine):
    """Empty records, records shorter than the primers, exact 64-base multiples, all-N, lower case."""
    recs = ["", "A", "ACG", "ACGTACGTAC" * 6 + "ACGT", "N" * 100, "acgtagctagctgatcgatgctagctagctgatcgat" * 5,
            "ACGT" * 16, "ACGT" * 16 + "A", "ACGT" * 16 + "ACG", "TTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTT" * 3, ""]
    wl = synth.random_small(1, n_records=1, len_lo=10, len_hi=10, n_pairs=1, plant=0)
    wl.seq = np.frombuffer("".join(recs).encode(), dtype=np.uint8).copy()
    wl.offsets = np.cumsum([0] + [len(r) for r in recs]).astype(np.int64)
    wl.genome_ids = np.arange(len(recs), dtype=np.uint32)
    for fwd, rev, k, clamp in [("ACGTA", "TACGT", 0, 0), ("ACGTA", "TACGT", 1, 5), ("AGCTAGCTGATC", "GATCGATG", 3, 2),
                               ("TTTTTTTT", "AAAAAAAA", 2, 3), ("NN", "AC", 0, 1), ("ACGTACGTACGTACGTACGTACGTACGTACGT",
                                                                                 "TTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTT", 15, 3)]:
        wl.fwd, wl.rev, wl.k, wl.clamp = [fwd], [rev], [k], clamp
        wl.min_len, wl.max_len, wl.fb_len, wl.rb_len, wl.trim = 1, 500, 7, 9, True
        _run_both(engine, wl)


def test_dense_sites_overflow_retry(engine):
    """Every window of a homopolymer run is a site: tiles overflow their slot lists and are re-run."""
    g = "A" * 300_000 + "ACGT" * 1000 + "T" * 200_000
    wl = synth.random_small(2, n_records=1, len_lo=10, len_hi=10, n_pairs=1, plant=0)
    wl.seq = np.frombuffer(g.encode(), dtype=np.uint8).copy()
    wl.offsets = np.array([0, len(g)], dtype=np.int64)
    wl.fwd, wl.rev, wl.k, wl.clamp = ["AAAAAAAAAA"], ["AAAAAAAAAAAA"], [1], 2
    wl.min_len, wl.max_len, wl.orient_mask = 20, 60, 15
    wl.fb_len = wl.rb_len = 3
    out, ref = _run_both(engine, wl)
    assert len(ref.hits) > 500_000


@pytest.mark.parametrize("threads,gpt,slots,shift", [(256, 4, 256, 1), (256, 4, 256, 2), (128, 1, 16, 0),
                                                     (512, 8, 64, 2), (64, 16, 4096, 1)])
def test_scan_shapes_and_shift_modes(engine, threads, gpt, slots, shift):
    """Every kernel shape and pattern-alignment mode gives the same sites (tiny slot lists force the
    overflow re-run)."""
    from paper_2511_00170_gb300 import ah

    ah.ah_ctx_set_scan_config(engine.ctx, threads, gpt, slots, shift)
    try:
        _run_both(engine, synth.batched(n_genomes=12, len_lo=2e3, len_hi=3e5, n_pairs=3))
        _run_both(engine, _random_case(1000 + threads + gpt + shift))
    finally:
        ah.ah_ctx_set_scan_config(engine.ctx, 256, 4, 256, 0)


@pytest.mark.parametrize("min_blocks,windows,queue", [(0, 1, 0), (0, 64, 1), (4, 4096, 0), (0, 1 << 20, 1),
                                                      (8, 1024, 1), (4, 4096, 1)])
def test_scan_circuit_splits(engine, min_blocks, windows, queue):
    """The circuit's phase split drawn for any number of windows per vote (1: the shortest first
    phase, 2^20: one phase for most patterns), any register bound, and candidates emitted where
    found or queued per warp give the same sites."""
    from paper_2511_00170_gb300 import ah

    ah.ah_ctx_set_scan_circuit(engine.ctx, min_blocks, windows, queue)
    try:
        _run_both(engine, synth.batched(n_genomes=12, len_lo=2e3, len_hi=3e5, n_pairs=4))
        _run_both(engine, _random_case(2000 + windows % 97 + min_blocks + queue))
    finally:
        ah.ah_ctx_set_scan_circuit(engine.ctx, 0, 1024, 0)


def test_candidate_queue_overflow(engine):
    """A site at every position: each warp's candidate queue overflows and the rest of its words are
    emitted where found; the sites still match the oracle's."""
    from paper_2511_00170_gb300 import ah

    g = "A" * 200_000 + "ACGT" * 500 + "T" * 100_000
    wl = synth.random_small(3, n_records=1, len_lo=10, len_hi=10, n_pairs=1, plant=0)
    wl.seq = np.frombuffer(g.encode(), dtype=np.uint8).copy()
    wl.offsets = np.array([0, len(g)], dtype=np.int64)
    wl.fwd, wl.rev, wl.k, wl.clamp = ["AAAAAAAAAA"], ["AAAAAAAAAAAA"], [1], 2
    wl.min_len, wl.max_len, wl.orient_mask = 20, 60, 15
    wl.fb_len = wl.rb_len = 3
    ah.ah_ctx_set_scan_circuit(engine.ctx, 0, 1024, 1)
    try:
        out, ref = _run_both(engine, wl)
        assert len(ref.hits) > 300_000
    finally:
        ah.ah_ctx_set_scan_circuit(engine.ctx, 0, 1024, 0)


def test_several_pairs(engine):
    wl = synth.batched(n_genomes=40, len_lo=2e3, len_hi=2e5, n_pairs=8)
    _run_both(engine, wl)


def test_deterministic(engine):
    from paper_2511_00170_gb300.pipeline import Params

    wl = synth.plain_small(n_genomes=4, len_lo=200_000, len_hi=400_000)
    a = engine.run_workload(wl)
    b = engine.run_workload(wl)
    assert a.hits.tobytes() == b.hits.tobytes()
    assert a.amps.tobytes() == b.amps.tobytes()
    assert a.arena == b.arena


COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def test_tm_duplexes(engine):
    """Random duplexes, 2-32 nt, 0-5 mismatches anywhere (every internal and terminal table entry is
    reached), all salt methods."""
    from paper_2511_00170_gb300 import ah

    st = synth.Stream(synth.make_key(3, 901, 0))
    seqs, cseqs = [], []
    for _ in range(20000):
        L = st.randint(2, 32)
        s = "".join(st.choice("ACGT") for _ in range(L))
        c = [COMP[x] for x in s]
        for _ in range(st.randint(0, 5)):
            p = st.randint(0, L - 1)
            c[p] = st.choice([b for b in "ACGT" if b != COMP[s[p]]])
        seqs.append(s)
        cseqs.append("".join(c))
    worst = 0.0
    for method, na in [(5, 50.0), (0, 50.0), (1, 20.0), (2, 100.0), (3, 50.0), (4, 10.0), (6, 50.0)]:
        tmp = synth.TmParams(Na=na, saltcorr=method)
        got = ah.ah_tm_duplexes(engine.ctx, seqs, cseqs, ah.tm_params(Na=na, saltcorr=method))
        for s, c, g in zip(seqs, cseqs, got):
            r = oracle.tm_duplex(s, c, tmp)
            if r is None:
                assert math.isnan(g), (s, c)
            else:
                worst = max(worst, abs(g - r))
                assert abs(g - r) <= compare.TM_TOL, (s, c, g, r)
    assert worst <= compare.TM_TOL


# every salt method with the other cations and dNTPs; method 7 in its three regimes (monovalent
# ions dominating, mixed, Mg2+ dominating) and with Mg2+ alone; self-complementary mode
_TM_OPTION_CASES = [
    dict(Na=50.0, Mg=1.5, dNTPs=0.8, K=10.0, Tris=20.0, saltcorr=5),
    dict(Na=50.0, Mg=2.0, dNTPs=0.2, saltcorr=6),
    dict(Na=100.0, K=50.0, Tris=10.0, saltcorr=1),
    dict(Na=30.0, Mg=1.0, saltcorr=2),
    dict(Na=200.0, Mg=0.0, saltcorr=7),
    dict(Na=50.0, Mg=2.0, dNTPs=0.8, saltcorr=7),
    dict(Na=10.0, Mg=3.0, saltcorr=7),
    dict(Na=0.0, Mg=4.0, dNTPs=1.0, saltcorr=7),
    dict(Na=50.0, saltcorr=5, selfcomp=1, dnac1=250.0),
    dict(Na=50.0, Mg=2.0, saltcorr=7, selfcomp=1, dnac1=100.0),
]


@pytest.mark.parametrize("case", _TM_OPTION_CASES)
def test_tm_duplex_options(engine, case):
    """Duplex Tm under the remaining Tm_NN options: K+, Tris, Mg2+ and dNTPs with every salt method,
    salt method 7 (Owczarzy et al. 2008) in each of its regimes, and self-complementary duplexes."""
    from paper_2511_00170_gb300 import ah

    st = synth.Stream(synth.make_key(4, 902, 0))
    seqs, cseqs = [], []
    for _ in range(3000):
        L = st.randint(2, 32)
        s = "".join(st.choice("ACGT") for _ in range(L))
        c = [COMP[x] for x in s]
        for _ in range(st.randint(0, 3)):
            p = st.randint(0, L - 1)
            c[p] = st.choice([b for b in "ACGT" if b != COMP[s[p]]])
        seqs.append(s)
        cseqs.append("".join(c))
    got = ah.ah_tm_duplexes(engine.ctx, seqs, cseqs, ah.tm_params(**case))
    tmp = synth.TmParams(**case)
    for s, c, g in zip(seqs, cseqs, got):
        r = oracle.tm_duplex(s, c, tmp)
        if r is None:
            assert math.isnan(g), (s, c)
        else:
            assert abs(g - r) <= compare.TM_TOL, (s, c, g, r)


def test_pack_layout(engine):
    """Planes and invalid words against the layout in include/ah.h, read back from the device."""
    import torch

    from paper_2511_00170_gb300 import ah

    wl = synth.random_small(9, n_records=5, len_lo=0, len_hi=700, n_frac=0.05, alphabet="ACGTacgtRYN")
    batch = engine.pack(wl.seq, wl.offsets)
    try:
        v = ah.ah_batch_view_get(batch)
        n = v["n_groups"]

        class _Dev:
            def __init__(self, ptr, shape, typestr):
                self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3}

        planes = torch.as_tensor(_Dev(v["planes"], (n, 2), "<u4"), device="cuda").cpu().numpy()
        inval = torch.as_tensor(_Dev(v["invalid"], (n,), "<u4"), device="cuda").cpu().numpy()
        rg = torch.as_tensor(_Dev(v["rec_group"], (wl.n_records,), "<u8"), device="cuda").cpu().numpy()
    finally:
        ah.ah_batch_free(batch)
    code = {"A": 0, "C": 1, "T": 2, "G": 3}
    expect_lo = np.zeros(n * 32, dtype=np.uint8)
    expect_hi = np.zeros(n * 32, dtype=np.uint8)
    expect_inv = np.ones(n * 32, dtype=np.uint8)
    g = 0
    for r in range(wl.n_records):
        s = wl.record_str(r)
        assert rg[r] == g and g % 2 == 0
        for i, ch in enumerate(s):
            c = ch.upper()
            if c in code:
                expect_lo[g * 32 + i] = code[c] & 1
                expect_hi[g * 32 + i] = code[c] >> 1
                expect_inv[g * 32 + i] = 0
        g += (len(s) // 64 + 1) * 2   # at least one padding base after every record
    assert g == n
    bits = lambda w: np.unpackbits(w.astype("<u4").view(np.uint8), bitorder="little")
    assert np.array_equal(bits(planes[:, 0]), expect_lo)
    assert np.array_equal(bits(planes[:, 1]), expect_hi)
    assert np.array_equal(bits(inval), expect_inv)


def _degenerate_sites(seed, n, codes_lo, codes_hi):
    st = synth.Stream(synth.make_key(seed, 77, 1))
    prims, sites, ks, clamps = [], [], [], []
    for _ in range(n):
        L = st.randint(12, 26)
        p = synth.random_primer(st, L, st.randint(codes_lo, codes_hi), 0, "RYSWKMBDHVNNN")
        v = synth.concrete_variant(st, p)
        sites.append(synth.substitute(st, v, st.randint(0, 4)))
        prims.append(p)
        ks.append(st.randint(0, 5))
        clamps.append(st.randint(0, 4))
    return prims, sites, ks, clamps


def _check_sites(got, prims, sites, ks, clamps, prm):
    for i, (p, s, g) in enumerate(zip(prims, sites, got)):
        k = None if ks is None else ks[i]
        c = 0 if clamps is None else clamps[i]
        r = oracle.tm_site(p, s, prm, k=k, clamp=c)
        if r is None:
            assert math.isnan(g), (p, s, k, c, g)
        else:
            assert abs(g - r) <= compare.TM_TOL, (p, s, k, c, g, r)


@pytest.mark.parametrize("method,na", [(5, 50.0), (0, 50.0), (1, 20.0), (3, 50.0), (4, 10.0), (2, 200.0)])
def test_degenerate_site_tm_exact_max(engine, method, na):
    """Sites of primers with 7-9 degenerate codes (128 to 262,144 variants, many of them within the
    mismatch budget) take the chain method with mismatch-counting states on the GPU; the oracle
    enumerates every variant and keeps the qualifying ones."""
    from paper_2511_00170_gb300 import ah

    prims, sites, ks, clamps = _degenerate_sites(method, 30, 7, 9)
    got = ah.ah_tm_sites(engine.ctx, prims, sites, ah.tm_params(Na=na, saltcorr=method), k=ks, clamp=clamps)
    _check_sites(got, prims, sites, ks, clamps, synth.TmParams(Na=na, saltcorr=method))


def test_degenerate_site_tm_wide_mismatch_budget(engine):
    """Mismatch budgets of 6 to 12 (7 to 13 states per base) on primers with 8-10 degenerate codes:
    beyond the widths whose Viterbi states stay in registers, the chain method keeps them in
    per-thread arrays; both forms must give the oracle's exact maximum."""
    from paper_2511_00170_gb300 import ah

    prims, sites, _, clamps = _degenerate_sites(31, 24, 8, 10)
    st = synth.Stream(synth.make_key(31, 78, 1))
    ks = [st.randint(6, 12) for _ in prims]
    got = ah.ah_tm_sites(engine.ctx, prims, sites, ah.tm_params(), k=ks, clamp=clamps)
    _check_sites(got, prims, sites, ks, clamps, synth.TmParams())


@pytest.mark.parametrize("method,na", [(4, 10.0), (5, 50.0)])
def test_degenerate_site_tm_no_mismatch_limit(engine, method, na):
    """Without a mismatch limit every variant counts; where some variant's entropy sum could reach
    zero the chain method does not apply and the GPU enumerates (at most 2^20 variants)."""
    from paper_2511_00170_gb300 import ah

    prims, sites, _, _ = _degenerate_sites(100 + method, 12, 7, 9)
    got = ah.ah_tm_sites(engine.ctx, prims, sites, ah.tm_params(Na=na, saltcorr=method))
    _check_sites(got, prims, sites, None, None, synth.TmParams(Na=na, saltcorr=method))


def test_degenerate_site_tm_small_sets_and_method6(engine):
    """Up to 64 qualifying variants, and salt method 6 at any count, enumerate on the GPU too."""
    from paper_2511_00170_gb300 import ah

    prims, sites, ks, clamps = _degenerate_sites(11, 40, 0, 6)
    for method in (5, 6):
        got = ah.ah_tm_sites(engine.ctx, prims, sites, ah.tm_params(saltcorr=method), k=ks, clamp=clamps)
        _check_sites(got, prims, sites, ks, clamps, synth.TmParams(saltcorr=method))


@pytest.mark.parametrize("case", [dict(Na=50.0, Mg=2.0, dNTPs=0.8, saltcorr=7), dict(Na=10.0, Mg=3.0, saltcorr=7),
                                  dict(Na=50.0, saltcorr=5, selfcomp=1), dict(Na=50.0, Mg=1.5, saltcorr=4, selfcomp=1)])
def test_degenerate_site_tm_options(engine, case):
    """Degenerate sites under salt method 7 (enumerated: the correction depends on each variant's G/C
    content) and in self-complementary mode (the chain method carries the symmetry term)."""
    from paper_2511_00170_gb300 import ah

    prims, sites, ks, clamps = _degenerate_sites(21 + case["saltcorr"], 24, 0, 8)
    got = ah.ah_tm_sites(engine.ctx, prims, sites, ah.tm_params(**case), k=ks, clamp=clamps)
    _check_sites(got, prims, sites, ks, clamps, synth.TmParams(**case))


def test_degenerate_site_tm_work_bound(engine):
    """More than 2^20 qualifying variants under salt method 6 (no chain method) is refused with
    AH_ELIMIT, and the context stays usable."""
    from paper_2511_00170_gb300 import ah

    p, s = "N" * 11 + "ACGTTGCAA", "ACGTACGTACGTACGTTGCAA"[1:]
    with pytest.raises(ah.AhError) as e:
        ah.ah_tm_sites(engine.ctx, [p], [s], ah.tm_params(saltcorr=6))
    assert e.value.status == ah.AH_ELIMIT
    # 4^11 variants with a budget of 3 mismatches: 4,984 qualify; the chain method handles them
    got = ah.ah_tm_sites(engine.ctx, [p], [s], ah.tm_params(saltcorr=5), k=[3], clamp=[4])
    r = oracle.tm_site(p, s, synth.TmParams(saltcorr=5), k=3, clamp=4)
    assert abs(got[0] - r) <= compare.TM_TOL


@pytest.mark.parametrize("variants", [0, 1])
def test_dense_workload_small(engine, variants):
    """Tandem repeats and highly degenerate primers (dense sites, overflowing tiles, chain Tm), with
    the site Tm over every variant or over the site-matching ones."""
    import dataclasses

    wl = synth.dense(n_genomes=10, median=2e5, sigma=0.3)
    wl.fwd = ["NNRYTGACCGTAGSAN"[:16]]
    wl.rev = ["NAGYCGATWKSGNACT"[:16]]
    wl.tm = dataclasses.replace(wl.tm, variants=variants)
    _run_both(engine, wl)


@pytest.mark.parametrize("big", [False, True])
def test_pack_paths_agree(engine, big):
    """Every packing path gives the same planes: host records from pageable memory (pipelined copies
    into 16-byte aligned staging, aligned vector kernel), host records in page-locked memory read in
    place at odd offsets, device records at odd offsets, and streamed range packs from device and
    from page-locked host memory.  The large case has records longer than one 2^20-base item."""
    import torch

    from paper_2511_00170_gb300 import ah

    if big:
        wl = synth.plain_small(n_genomes=5, len_lo=1_100_000, len_hi=2_600_000)
    else:
        wl = synth.random_small(21, n_records=40, len_lo=0, len_hi=3000, n_frac=0.03, alphabet="ACGTacgtRYN", plant=0)
        # lengths around the 16-byte word and the 32-base group
        extra = [b"", b"A", b"ACGTACGTACGTACG", b"ACGTACGTACGTACGT", b"NACGTACGTACGTACGT", b"acgt" * 8 + b"N",
                 b"ACGT" * 16 + b"TT"]
        wl.seq = np.concatenate([wl.seq] + [np.frombuffer(x, np.uint8) for x in extra])
        wl.offsets = np.concatenate([wl.offsets, wl.offsets[-1] + np.cumsum([len(x) for x in extra])]).astype(np.int64)
        wl.genome_ids = np.arange(len(wl.offsets) - 1, dtype=np.uint32)

    class _Dev:
        def __init__(self, ptr, shape, typestr):
            self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3}

    def planes_of(batch):
        v = ah.ah_batch_view_get(batch)
        n = v["n_groups"]
        p = torch.as_tensor(_Dev(v["planes"], (n, 2), "<u4"), device="cuda").cpu().numpy().copy()
        i = torch.as_tensor(_Dev(v["invalid"], (n,), "<u4"), device="cuda").cpu().numpy().copy()
        return p, i

    n_rec = len(wl.offsets) - 1
    lengths = np.diff(wl.offsets).astype(np.uint64)
    host = engine.pack(wl.seq, wl.offsets)
    pinned = torch.empty(len(wl.seq) + 5, dtype=torch.uint8, pin_memory=True)
    pinned.numpy()[5:] = wl.seq
    in_place = engine.pack(pinned.numpy()[5:], wl.offsets)   # odd offsets in page-locked memory
    d = torch.from_numpy(np.concatenate([np.zeros(3, np.uint8), wl.seq])).cuda()   # unaligned records
    dev = engine.pack_device(d.data_ptr() + 3, wl.offsets.astype(np.uint64))
    ah.ah_ctx_synchronize(engine.ctx)
    streamed = ah.ah_batch_create(engine.ctx, lengths)
    streamed_host = ah.ah_batch_create(engine.ctx, lengths)
    half = n_rec // 2
    for a, b_ in ((0, half), (half, n_rec)):
        o = (wl.offsets[a:b_ + 1] - wl.offsets[a]).astype(np.uint64)
        ah.ah_batch_pack_range(engine.ctx, streamed, a, d.data_ptr() + 3 + int(wl.offsets[a]), o)
        ah.ah_batch_pack_range(engine.ctx, streamed_host, a, pinned.data_ptr() + 5 + int(wl.offsets[a]), o)
    try:
        ph, ih = planes_of(host)
        for other in (in_place, dev, streamed, streamed_host):
            po, io = planes_of(other)
            assert np.array_equal(ph, po) and np.array_equal(ih, io)
    finally:
        for x in (host, in_place, dev, streamed, streamed_host):
            ah.ah_batch_free(x)


@pytest.mark.parametrize("pairs_per_kernel", [1, 3])
def test_pairs_per_kernel(engine, pairs_per_kernel):
    """Scans split into kernels of a few pairs each (compiled in parallel, launched in turn into the
    same tile slot lists) give the oracle's outputs, as one kernel for every pair does."""
    from paper_2511_00170_gb300 import ah

    wl = synth.batched(n_genomes=24, len_lo=2e3, len_hi=2e5, n_pairs=7)
    ah.ah_ctx_set_pairs_per_kernel(engine.ctx, pairs_per_kernel)
    try:
        _run_both(engine, wl)
    finally:
        ah.ah_ctx_set_pairs_per_kernel(engine.ctx, 0)


def test_batch_export_import(engine):
    """A packed batch exported (dense planes, sparse invalid words) and imported into a fresh layout
    gives the same planes, invalid words and outputs; an index past the batch is refused."""
    import torch

    from paper_2511_00170_gb300 import ah

    wl = synth.random_small(23, n_records=30, len_lo=0, len_hi=4000, n_frac=0.03, alphabet="ACGTacgtRYN", plant=2)
    a = engine.pack(wl.seq, wl.offsets)
    b = ah.ah_batch_create(engine.ctx, wl.lengths().astype(np.uint64))
    try:
        planes, groups, words = ah.ah_batch_export(a)
        v = ah.ah_batch_view_get(a)
        assert planes.shape == (v["n_groups"], 2) and len(groups) == len(words) > 0
        ah.ah_batch_import(engine.ctx, b, planes, groups, words)
        p2, g2, w2 = ah.ah_batch_export(b)
        assert np.array_equal(planes, p2) and np.array_equal(groups, g2) and np.array_equal(words, w2)
        from paper_2511_00170_gb300.pipeline import Params

        p = Params.from_workload(wl)
        o1, o2 = engine.step(a, p), engine.step(b, p)
        assert o1.hits.tobytes() == o2.hits.tobytes() and o1.amps.tobytes() == o2.amps.tobytes()
        assert o1.arena == o2.arena
        bad = groups.copy()
        bad[0] = v["n_groups"]
        with pytest.raises(ah.AhError) as e:
            ah.ah_batch_import(engine.ctx, b, planes, bad, words)
        assert e.value.status == ah.AH_EINVAL
    finally:
        ah.ah_batch_free(a)
        ah.ah_batch_free(b)


@pytest.fixture(params=[1, 3], ids=["generic", "handover"])
def generic(engine, request):
    """The engine's context with the generic (compile-free) scan kernel forced over every tile, or
    over the first half of the tiles with the generated kernels on the rest."""
    from paper_2511_00170_gb300 import ah

    ah.ah_ctx_set_generic_scan(engine.ctx, request.param)
    ah.ah_ctx_stats_reset(engine.ctx)
    try:
        yield engine
        if request.param == 1:
            assert ah.ah_ctx_stats_get(engine.ctx)["generic_scans"] > 0
    finally:
        ah.ah_ctx_set_generic_scan(engine.ctx, 0)


@pytest.mark.parametrize("seed", range(24))
def test_generic_scan_random_small(generic, seed):
    """The generic kernel (primer set read from a table at run time) finds the oracle's sites."""
    _run_both(generic, _random_case(seed))


def test_generic_scan_edges_and_overflow(generic):
    """Edge records, degenerate primers up to 32 bases with k = 15, and the dense-tile re-run, through
    the generic kernel."""
    test_edge_records(generic)
    test_dense_sites_overflow_retry(generic)


@pytest.mark.parametrize("threads,gpt,slots", [(128, 8, 256), (256, 4, 64), (64, 16, 16)])
def test_generic_scan_many_pairs(generic, threads, gpt, slots):
    """Twenty pairs: more patterns than one generic launch holds (64), so two launches append to the
    same tile slot lists; every tile shape."""
    from paper_2511_00170_gb300 import ah

    ah.ah_ctx_set_scan_config(generic.ctx, threads, gpt, slots, 0)
    try:
        _run_both(generic, synth.batched(n_genomes=16, len_lo=2e3, len_hi=2e5, n_pairs=20))
    finally:
        ah.ah_ctx_set_scan_config(generic.ctx, 256, 4, 256, 0)


def test_generic_scan_auto(engine):
    """Mode 2 starts a primer set whose kernels are not compiled on the generic kernel, compiling them
    on a thread of the context (not waited for by a scan the generic kernel finishes first); once
    they are compiled, it scans with them."""
    from paper_2511_00170_gb300 import ah

    wl = synth.random_small(7_770_001, n_records=3, len_lo=500, len_hi=3000, n_pairs=2, plen_lo=17, plen_hi=23,
                            n_deg=3, k_max=3, clamp=2, plant=3)
    ctx = engine.ctx
    ah.ah_ctx_set_generic_scan(ctx, 2)
    try:
        ah.ah_ctx_stats_reset(ctx)
        _run_both(engine, wl)
        s = ah.ah_ctx_stats_get(ctx)
        assert s["generic_scans"] >= 1   # the second step may find them compiled
        ah.ah_ctx_set_generic_scan(ctx, 0)
        _run_both(engine, wl)                                        # waits for the compile if still running
        ah.ah_ctx_set_generic_scan(ctx, 2)
        ah.ah_ctx_stats_reset(ctx)
        _run_both(engine, wl)
        s = ah.ah_ctx_stats_get(ctx)
        assert s["generic_scans"] == 0 and s["generic_bases"] == 0 and s["jit_compiles"] == 0
    finally:
        ah.ah_ctx_set_generic_scan(ctx, 0)


@pytest.fixture(scope="module")
def near_case():
    """A small planted workload and the oracle's unfiltered result (Tm does not depend on min_tm)."""
    wl = synth.plain_small(n_genomes=4, len_lo=200_000, len_hi=400_000)
    wl.tm.min_tm = None
    ref = oracle.run(wl, with_seqs=False)
    defined = np.nonzero(ref.amp_status == 0)[0]
    assert len(defined) > 0
    return wl, ref, float(ref.amp_tm[defined[0]])


@pytest.mark.parametrize("offset", [0.0, 5e-10, -5e-10, 2e-9, -2e-9])
def test_near_threshold_flags(engine, near_case, offset):
    """min_tm at an amplicon's exact oracle Tm, then 5e-10 and 2e-9 C to either side.  Flags bit1 must
    mark exactly the amplicons within 1e-9 C of min_tm, bit0 the threshold decision; both with the
    filter on (kept list) and off (every amplicon annotated)."""
    import dataclasses

    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Params

    wl, ref_u, t0 = near_case
    thr = t0 + offset
    ref = dataclasses.replace(ref_u, keep=oracle.tm_keep(ref_u.amp_tm, ref_u.amp_status, thr),
                              near=oracle.tm_near(ref_u.amp_tm, ref_u.amp_status, thr), min_tm=thr)
    near_expected = abs(offset) <= 1e-9
    assert ref.near.any() == near_expected
    batch = engine.pack(wl.seq, wl.offsets, wl.genome_ids)
    try:
        p = Params.from_workload(wl)
        p.min_tm = thr
        out_f = engine.step(batch, p, with_seqs=False)
        p.filter = False
        out_a = engine.step(batch, p, with_seqs=False)
    finally:
        ah.ah_batch_free(batch)
    compare.assert_same_amplicons(out_f, ref, filtered=True, min_tm=thr)
    compare.assert_same_amplicons(out_a, ref, filtered=False, min_tm=thr)
    # the annotated list holds every amplicon: the flagged ones are exactly the oracle's near ones,
    # and away from the exact Tm the decision is the oracle's
    flagged = (out_a.amps["flags"] & 2) != 0
    assert int(flagged.sum()) == int(ref.near.sum())
    t_gpu = out_a.amps["tm"][flagged]
    assert np.all(np.abs(t_gpu - thr) <= 1e-9)
    if offset != 0.0:
        dec = (out_a.amps["flags"] & 1) != 0
        assert int(dec.sum()) == int(ref.keep.sum())
        assert len(out_f.amps) == int(ref.keep.sum())
