"""Pins for the oracle's scan (Supplementary, "Primer matching and clamp logic").

The oracle counts mismatches per position against IUPAC sets.  These tests check it against
(1) brute-force enumeration of every concrete primer variant with plain character comparison,
(2) exact substring search when k=0 and the primers are plain ACGT,
(3) the reverse-complement bijection of sites, and (4) planted-site truth from the generator.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import brute


def _oracle_tuples(hits):
    return [(int(h["record"]), int(h["pair"]), int(h["pos"]), int(h["strand"]), int(h["primer"]), int(h["mism"]))
            for h in hits]


@pytest.mark.parametrize("seed", list(range(12)))
def test_scan_matches_bruteforce_variants(seed):
    wl = synth.random_small(seed, n_records=3, len_lo=0, len_hi=160, n_pairs=2, plen_lo=4, plen_hi=8, n_deg=3,
                            k_max=3, clamp=seed % 3, n_frac=0.03, alphabet="ACGT" if seed % 2 else "ACGTACGTacgt")
    records = [wl.record_str(i) for i in range(wl.n_records)]
    expect = brute.scan(records, wl.fwd, wl.rev, wl.k, wl.clamp)
    got = _oracle_tuples(oracle.scan(wl, threads=2))
    assert got == expect


@pytest.mark.parametrize("seed", [100, 101, 102])
def test_scan_low_complexity_bruteforce(seed):
    # a two-letter genome makes many overlapping near-hits
    wl = synth.random_small(seed, n_records=2, len_lo=80, len_hi=200, n_pairs=1, plen_lo=5, plen_hi=7, n_deg=2,
                            k_max=2, clamp=1, n_frac=0.0, alphabet="AT", plant=0)
    records = [wl.record_str(i) for i in range(wl.n_records)]
    assert _oracle_tuples(oracle.scan(wl)) == brute.scan(records, wl.fwd, wl.rev, wl.k, wl.clamp)


def test_k0_plain_primers_is_substring_search():
    wl = synth.random_small(7, n_records=4, len_lo=300, len_hi=600, n_pairs=1, plen_lo=3, plen_hi=4, n_deg=0,
                            k_max=0, clamp=0, n_frac=0.0, plant=2)
    wl.k = [0]
    rc = str.maketrans("ACGT", "TGCA")
    expect = []
    for r in range(wl.n_records):
        g = wl.record_str(r).upper()
        for primer, P in ((0, wl.fwd[0]), (1, wl.rev[0])):
            for strand, pat in ((0, P), (1, P.translate(rc)[::-1])):
                i = g.find(pat)
                while i >= 0:
                    expect.append((r, 0, i, strand, primer, 0))
                    i = g.find(pat, i + 1)
    expect.sort(key=lambda h: (h[0], h[1], h[2], h[3], h[4]))
    assert _oracle_tuples(oracle.scan(wl)) == expect
    assert len(expect) > 0


def _revcomp_record(s: str) -> str:
    t = str.maketrans("ACGTacgt", "TGCAtgca")
    return s.translate(t)[::-1]


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_scan_reverse_complement_bijection(seed):
    """Scanning rc(G) gives the mirrored sites: [p,p+L) on strand s <-> [len-p-L, len-p) on 1-s."""
    wl = synth.random_small(seed, n_records=3, len_lo=200, len_hi=400, n_pairs=2, plen_lo=6, plen_hi=9, n_deg=3,
                            k_max=3, clamp=2, n_frac=0.02)
    rc_wl = wl.subset(range(wl.n_records))
    for r in range(wl.n_records):
        a, b = rc_wl.offsets[r], rc_wl.offsets[r + 1]
        rc_wl.seq[a:b] = np.frombuffer(_revcomp_record(wl.record_str(r)).encode(), dtype=np.uint8)
    h = oracle.scan(wl)
    hr = oracle.scan(rc_wl)
    lens = wl.lengths()

    def L(x):
        return len(wl.fwd[x["pair"]] if x["primer"] == 0 else wl.rev[x["pair"]])

    mapped = sorted((int(x["record"]), int(x["pair"]), int(lens[x["record"]] - x["pos"] - L(x)), 1 - int(x["strand"]),
                     int(x["primer"]), int(x["mism"])) for x in h)
    assert mapped == sorted(_oracle_tuples(hr))
    assert len(h) > 0


def test_planted_exact_sites_are_found():
    """Planted templates whose binding sites carry no substitution must be hits (clamp intact)."""
    wl = synth.plain_small(n_genomes=3, len_lo=20000, len_hi=30000)
    hits = oracle.scan(wl)
    have = {(int(h["record"]), int(h["pos"]), int(h["primer"]), int(h["strand"])) for h in hits}
    lf, lr = len(wl.fwd[0]), len(wl.rev[0])
    n = 0
    for p in wl.planted:
        if p.subs_f == 0:
            # F site at the template start (top strand) or, when the template was reverse
            # complemented, at its end on the - strand
            key = (p.genome, p.pos, 0, 0) if p.strand == 0 else (p.genome, p.pos + p.length - lf, 0, 1)
            assert key in have
            n += 1
        if p.subs_r == 0:
            key = (p.genome, p.pos + p.length - lr, 1, 1) if p.strand == 0 else (p.genome, p.pos, 1, 0)
            assert key in have
            n += 1
    assert n > 0


def test_invalid_windows_and_bounds():
    # N inside a window removes the site; a site touching the record end is still found
    wl = synth.random_small(1, n_records=1, len_lo=30, len_hi=30, n_pairs=1, plen_lo=5, plen_hi=5, n_deg=0, k_max=0,
                            clamp=0, n_frac=0.0, plant=0)
    wl.fwd, wl.rev, wl.k = ["ACGTA"], ["GGGGG"], [0]
    g = list("TTTTTTTTTTACGTATTTTTACNTATTACGTA")
    wl.seq = np.frombuffer("".join(g).encode(), dtype=np.uint8).copy()
    wl.offsets = np.array([0, len(g)], dtype=np.int64)
    hits = _oracle_tuples(oracle.scan(wl))
    assert (0, 0, 10, 0, 0, 0) in hits
    assert (0, 0, len(g) - 5, 0, 0, 0) in hits
    assert not any(h[2] == 20 for h in hits)


def test_check_primer_validation():
    assert oracle.check_primer("ACGTRYKMSWBDHVN", 3, 2) == 0
    assert oracle.check_primer("ACGU", 1, 0) == 1
    assert oracle.check_primer("A" * 33, 1, 0) == 2
    assert oracle.check_primer("ACGT", 5, 0) == 3
    assert oracle.check_primer("ACGT", 1, 5) == 4


@pytest.mark.parametrize("seed", [40, 41])
def test_scan_output_does_not_depend_on_threads(seed):
    """The oracle splits records across threads for speed; its sites, in canonical order, are the
    same for any number of threads."""
    wl = synth.random_small(seed, n_records=23, len_lo=0, len_hi=3000, n_pairs=3, plen_lo=6, plen_hi=12, n_deg=3,
                            k_max=3, clamp=2, n_frac=0.01, plant=2)
    one = oracle.scan(wl, threads=1)
    assert len(one) > 0
    for t in (3, 7):
        assert np.array_equal(oracle.scan(wl, threads=t), one)
