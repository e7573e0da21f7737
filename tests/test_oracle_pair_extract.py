"""Pins for the oracle's pairing and extraction (Supplementary, "Amplicon calling and
orientation", "Primer trimming and barcode extraction").

Hand-built site layouts check each pairing reading; the reverse-complement identity checks
pairing, orientation, the RF reverse complement, trimming and the barcode sides together.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import brute


class _WL:
    """Minimal stand-in carrying what oracle.pair needs."""

    def __init__(self, lf, lr, min_len, max_len, mask=0b1111):
        self.fwd = ["A" * x for x in lf]
        self.rev = ["A" * x for x in lr]
        self.min_len, self.max_len, self.orient_mask = min_len, max_len, mask


def _hits(rows):
    """rows: (record, pair, pos, strand, primer) in the oracle's sorted order."""
    h = np.zeros(len(rows), dtype=oracle.HIT_DTYPE)
    for i, (r, p, pos, s, x) in enumerate(rows):
        h[i]["record"], h[i]["pair"], h[i]["pos"], h[i]["strand"], h[i]["primer"] = r, p, pos, s, x
    order = np.lexsort((h["primer"], h["strand"], h["pos"], h["pair"], h["record"]))
    return h[order]


def _amps(wl, rows, mask=None):
    a = oracle.pair(wl, _hits(rows), mask)
    return [(int(x["record"]), int(x["pair"]), int(x["start"]), int(x["end"]), oracle.ORIENT_NAMES[x["orient"]])
            for x in a]


F, R = 0, 1
P, M = 0, 1   # + and - strand

CASES = [
    # simple FR: F+ at 10, R- at 100 (L=20): [10, 120)
    ([(0, 0, 10, P, F), (0, 0, 100, M, R)], [(0, 0, 10, 120, "FR")]),
    # a same-sense site stops the walk: only the inner anchor pairs
    ([(0, 0, 10, P, F), (0, 0, 50, P, F), (0, 0, 100, M, R)], [(0, 0, 50, 120, "FR")]),
    # every antisense site before the stop pairs (reading R6)
    ([(0, 0, 10, P, F), (0, 0, 100, M, R), (0, 0, 200, M, R)], [(0, 0, 10, 120, "FR"), (0, 0, 10, 220, "FR")]),
    # too long: the walk stops at the first site beyond max (and does not resume)
    ([(0, 0, 10, P, F), (0, 0, 3000, M, R), (0, 0, 3010, M, F)], []),
    # too short: skipped, the walk continues
    ([(0, 0, 10, P, F), (0, 0, 15, M, R), (0, 0, 100, M, R)], [(0, 0, 10, 120, "FR")]),
    # orientations
    ([(0, 0, 10, P, R), (0, 0, 100, M, F)], [(0, 0, 10, 120, "RF")]),
    ([(0, 0, 10, P, F), (0, 0, 100, M, F)], [(0, 0, 10, 120, "FF")]),
    ([(0, 0, 10, P, R), (0, 0, 100, M, R)], [(0, 0, 10, 120, "RR")]),
    # ties at one position: + before -; the R+ at 10 stops F+ at 10
    ([(0, 0, 10, P, F), (0, 0, 10, P, R), (0, 0, 100, M, R)], [(0, 0, 10, 120, "RR")]),
    # records and pairs do not interact
    ([(0, 0, 10, P, F), (1, 0, 100, M, R), (0, 1, 100, M, R)], []),
    # exact window ends are inclusive (min 50 .. max 2000)
    ([(0, 0, 0, P, F), (0, 0, 30, M, R)], [(0, 0, 0, 50, "FR")]),
    ([(0, 0, 0, P, F), (0, 0, 1980, M, R)], [(0, 0, 0, 2000, "FR")]),
    ([(0, 0, 0, P, F), (0, 0, 1981, M, R)], []),
    # antisense site left of every anchor: unpaired
    ([(0, 0, 5, M, R), (0, 0, 100, P, F)], []),
]


@pytest.mark.parametrize("rows,expect", CASES)
def test_pairing_cases(rows, expect):
    wl = _WL([20, 20], [20, 20], 50, 2000)
    assert _amps(wl, rows) == expect


def test_orientation_mask_filters_after_pairing():
    wl = _WL([20], [20], 50, 2000)
    rows = [(0, 0, 10, P, F), (0, 0, 100, M, F), (0, 0, 200, M, R)]
    assert _amps(wl, rows, 0b1111) == [(0, 0, 10, 120, "FF"), (0, 0, 10, 220, "FR")]
    # FF is removed but the walk still reaches the FR partner (reading R9)
    assert _amps(wl, rows, 0b0011) == [(0, 0, 10, 220, "FR")]


def test_walk_stops_at_first_site_beyond_max():
    # R- at 1985 (L=20) ends at 2005 > max; the later F- at 1990 (L=5) would end inside the window,
    # but the walk has already stopped (reading R6)
    wl = _WL([5], [20], 50, 2000)
    assert _amps(wl, [(0, 0, 0, P, F), (0, 0, 1985, M, R), (0, 0, 1990, M, F)]) == []
    assert _amps(wl, [(0, 0, 0, P, F), (0, 0, 1990, M, F)]) == [(0, 0, 0, 1995, "FF")]


def test_primer_lengths_enter_the_end():
    wl = _WL([18], [25], 10, 2000)
    assert _amps(wl, [(0, 0, 10, P, F), (0, 0, 100, M, R)]) == [(0, 0, 10, 125, "FR")]
    assert _amps(wl, [(0, 0, 10, P, R), (0, 0, 100, M, F)]) == [(0, 0, 10, 118, "RF")]


def _rc_workload(wl):
    t = str.maketrans("ACGTacgt", "TGCAtgca")
    out = wl.subset(range(wl.n_records))
    for r in range(wl.n_records):
        a, b = out.offsets[r], out.offsets[r + 1]
        out.seq[a:b] = np.frombuffer(wl.record_str(r).translate(t)[::-1].encode(), dtype=np.uint8)
    return out


@pytest.mark.parametrize("seed", [11, 12, 13, 14])
def test_reverse_complement_identity(seed):
    """Pairing rc(G) with the oracle == the mirrored rule on G's own sites, with FR<->RF swapped and
    identical amplicon sequences, trimmed sequences and barcodes."""
    wl = synth.random_small(seed, n_records=3, len_lo=150, len_hi=400, n_pairs=2, plen_lo=6, plen_hi=9, n_deg=2,
                            k_max=2, clamp=2, n_frac=0.02, plant=3, min_len=10, max_len=150, fb=4, rb=6)
    rcw = _rc_workload(wl)
    hits = oracle.scan(wl)
    hr = oracle.scan(rcw)
    ar = oracle.pair(rcw, hr)
    lens = wl.lengths()

    def L(h):
        return len(wl.fwd[h["pair"]] if h["primer"] == 0 else wl.rev[h["pair"]])

    mir = brute.pair_mirrored([dict(record=int(h["record"]), pair=int(h["pair"]), pos=int(h["pos"]),
                                    strand=int(h["strand"]), primer=int(h["primer"])) for h in hits],
                              lambda h: L(h), lens, wl.min_len, wl.max_len)
    # rc(G) amplicons mapped back to G coordinates
    back = sorted((int(a["record"]), int(a["pair"]), int(lens[a["record"]] - a["end"]), int(lens[a["record"]] - a["start"]))
                  for a in ar)
    assert back == sorted(m[:4] for m in mir)
    assert len(mir) > 0
    # sequences: build G-side amplicons from the mirrored pairs and extract them
    swap = {0: 1, 1: 0, 2: 2, 3: 3}   # FR<->RF; FF and RR map to themselves
    g_amps = np.zeros(len(mir), dtype=oracle.AMP_DTYPE)
    for i, (r, p, s, e, ip, im) in enumerate(mir):
        g_amps[i]["record"], g_amps[i]["pair"], g_amps[i]["start"], g_amps[i]["end"] = r, p, s, e
        g_amps[i]["hit_i"], g_amps[i]["hit_j"] = ip, im
        xi, xj = int(hits[ip]["primer"]), int(hits[im]["primer"])
        g_amps[i]["orient"] = {(0, 1): 0, (1, 0): 1, (0, 0): 2, (1, 1): 3}[(xi, xj)]
    for trim in (False, True):
        ex_g = oracle.extract(wl, hits, g_amps, trim=trim)
        ex_r = oracle.extract(rcw, hr, ar, trim=trim)
        key_g = {}
        for a, x in zip(g_amps, ex_g):
            key_g[(int(a["record"]), int(a["pair"]), int(a["start"]), int(a["end"]))] = (int(a["orient"]), x)
        for a, x in zip(ar, ex_r):
            r = int(a["record"])
            k = (r, int(a["pair"]), int(lens[r] - a["end"]), int(lens[r] - a["start"]))
            og, xg = key_g[k]
            assert swap[og] == int(a["orient"])
            if og in (0, 1):   # FR on one side is RF on the other: same sequence and barcodes
                assert xg[:3] == x[:3]
            else:              # FF/RR stay on the top strand: the sequences are reverse complements
                t = str.maketrans("ACGTN", "TGCAN")
                assert xg[0] == x[0].translate(t)[::-1]


def test_extract_hand_example():
    # 0         1         2         3         4
    # 0123456789012345678901234567890123456789012
    g = "TTGCAACGTAGGCTTTCCCAAAGGGTTTGCATGCANNCGTAC"
    wl = synth.random_small(0, n_records=1, len_lo=10, len_hi=10, n_pairs=1, plant=0)
    wl.seq = np.frombuffer(g.encode(), dtype=np.uint8).copy()
    wl.offsets = np.array([0, len(g)], dtype=np.int64)
    wl.fwd, wl.rev = ["ACGTA"], ["TGCAA"]       # lengths 5 and 5
    hits = _hits([(0, 0, 5, P, F), (0, 0, 27, M, R)])
    hits = hits.copy()
    amps = np.zeros(2, dtype=oracle.AMP_DTYPE)
    # FR over [5, 32) and the same sites called as RF
    for i, o in enumerate((0, 1)):
        amps[i]["record"], amps[i]["start"], amps[i]["end"], amps[i]["hit_i"], amps[i]["hit_j"], amps[i]["orient"] = \
            0, 5, 32, 0, 1, o
    fr, rf = oracle.extract(wl, hits, amps, trim=False, fb=3, rb=4)
    assert fr[0] == g[5:32]
    assert fr[1] == g[2:5] and fr[2] == "GCAN"          # N stays N (reading R12)
    assert fr[3] == g[5:10]
    rcm = lambda s: s.translate(str.maketrans("ACGTN", "TGCAN"))[::-1]
    assert fr[4] == rcm(g[27:32])
    assert rf[0] == rcm(g[5:32])
    assert rf[1] == rcm(g[32:35]) and rf[2] == rcm(g[1:5])
    trimmed = oracle.extract(wl, hits, amps, trim=True, fb=0, rb=0)
    assert trimmed[0][0] == g[10:27] and trimmed[1][0] == rcm(g[10:27])
    # clipping at the record ends (reading R12)
    far = oracle.extract(wl, hits, amps, trim=False, fb=50, rb=50)
    assert far[0][1] == g[0:5] and far[0][2] == g[32:]


def test_trim_overlapping_sites_is_empty():
    wl = _WL([20], [20], 1, 2000)
    g = "ACGT" * 20
    wl2 = synth.random_small(0, n_records=1, len_lo=10, len_hi=10, n_pairs=1, plant=0)
    wl2.seq = np.frombuffer(g.encode(), dtype=np.uint8).copy()
    wl2.offsets = np.array([0, len(g)], dtype=np.int64)
    wl2.fwd, wl2.rev = wl.fwd, wl.rev
    hits = _hits([(0, 0, 10, P, F), (0, 0, 15, M, R)])
    a = oracle.pair(_WL([20], [20], 1, 2000), hits)
    assert len(a) == 1
    (x,) = oracle.extract(wl2, hits, a, trim=True, fb=0, rb=0)
    assert x[0] == ""


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_amplicon_qualities_follow_the_sequences(seed):
    """Given each record's own bases as its qualities, an amplicon's quality field is its sequence
    field for FR, FF and RR, and the complement of it for RF (qualities are reversed with the bases
    but not complemented), trimmed or not."""
    wl = synth.random_small(seed, n_records=3, len_lo=150, len_hi=400, n_pairs=2, plen_lo=6, plen_hi=9, n_deg=2,
                            k_max=2, clamp=2, n_frac=0.0, plant=3, min_len=10, max_len=150, fb=0, rb=0)
    hits = oracle.scan(wl)
    amps = oracle.pair(wl, hits)
    assert len(amps) > 0 and 1 in set(int(o) for o in amps["orient"])
    quals = [wl.record_str(r).upper().encode() for r in range(wl.n_records)]
    comp = bytes.maketrans(b"ACGT", b"TGCA")
    for trim in (False, True):
        wl.trim = trim
        got = oracle.amplicon_qualities(wl, hits, amps, quals)
        ex = oracle.extract(wl, hits, amps, trim=trim)
        for a, q, x in zip(amps, got, ex):
            s = x[0].upper().encode()
            assert q == (s.translate(comp) if int(a["orient"]) == 1 else s), (int(a["orient"]), trim)
