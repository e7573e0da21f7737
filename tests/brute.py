"""Brute-force restatements used to pin the oracle on tiny inputs.

These avoid every shortcut the oracle takes: primers are expanded into all their concrete
ACGT variants first (IUPAC sets written out here independently), each variant's reverse
complement is taken on the concrete string, and matching is plain character comparison.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Tuple

EXPAND = {"A": "A", "C": "C", "G": "G", "T": "T", "R": "AG", "Y": "CT", "S": "GC", "W": "AT", "K": "GT",
          "M": "AC", "B": "CGT", "D": "AGT", "H": "ACT", "V": "ACG", "N": "ACGT"}
_RC = str.maketrans("ACGT", "TGCA")


def variants(primer: str) -> List[str]:
    return ["".join(v) for v in itertools.product(*[EXPAND[c] for c in primer.upper()])]


def rc_concrete(s: str) -> str:
    return s.translate(_RC)[::-1]


def scan(records: List[str], fwd: List[str], rev: List[str], ks: List[int], clamp: int) -> List[Tuple]:
    """Hits as tuples (record, pair, pos, strand, primer, mism), sorted.

    A site is a hit iff some concrete variant v of the primer (v itself on the + strand, its
    reverse complement on the - strand) agrees with the genome at every clamp position (the
    primer's 3' end) and differs at no more than k positions; mism is the minimum over those
    variants.  Windows with a character outside ACGT (after upper-casing) are skipped.
    """
    out = []
    for r, g in enumerate(records):
        G = g.upper()
        for pr in range(len(fwd)):
            for primer, P in ((0, fwd[pr]), (1, rev[pr])):
                L = len(P)
                vs = variants(P)
                for strand in (0, 1):
                    pats = vs if strand == 0 else [rc_concrete(v) for v in vs]
                    clamp_idx = range(L - clamp, L) if strand == 0 else range(0, clamp)
                    for p in range(0, len(G) - L + 1):
                        w = G[p:p + L]
                        if any(ch not in "ACGT" for ch in w):
                            continue
                        best = None
                        for v in pats:
                            if any(v[j] != w[j] for j in clamp_idx):
                                continue
                            mm = sum(1 for a, b in zip(v, w) if a != b)
                            if best is None or mm < best:
                                best = mm
                        if best is not None and best <= ks[pr]:
                            out.append((r, pr, p, strand, primer, best))
    out.sort(key=lambda h: (h[0], h[1], h[2], h[3], h[4]))
    return out


def pair_mirrored(hits: List[Dict], len_of, rec_len, min_len: int, max_len: int) -> List[Tuple]:
    """The oracle's pairing rule applied to the reverse complement of each record, written in the
    record's own coordinates.  Reverse-complementing maps a site at [p, p+L) on strand s to
    [len-p-L, len-p) on strand 1-s, so here the sites are ordered by decreasing end (ties: - strand
    first, then F before R), anchors are the - strand sites, and a - strand site stops the walk.
    Returns (record, pair, start, end, index of the + site, index of the - site)."""
    out = []
    by = {}
    for idx, h in enumerate(hits):
        by.setdefault((h["record"], h["pair"]), []).append((idx, h))
    for key, hs in by.items():
        hs.sort(key=lambda t: (-(t[1]["pos"] + len_of(t[1])), 1 - t[1]["strand"], t[1]["primer"]))
        for a in range(len(hs)):
            ia, A = hs[a]
            if A["strand"] != 1:
                continue
            end = A["pos"] + len_of(A)
            for b in range(a + 1, len(hs)):
                ib, B = hs[b]
                if B["strand"] == 1:
                    break
                length = end - B["pos"]
                if length > max_len:
                    break
                if length < min_len:
                    continue
                out.append((key[0], key[1], B["pos"], end, ib, ia))
    return sorted(out)
