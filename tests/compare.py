"""Helpers that put the CUDA path's outputs and the oracle's into one comparable form.

The CUDA path orders hits by (pair, record, pos, orient) and amplicons by (anchor, partner);
the oracle orders by (record, pair, pos, strand, primer).  Both are unique orders of the same
sets, so comparisons sort both sides by the same keys and compare element by element.
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np

TM_TOL = 1e-9  # degrees C


def gpu_hit_tuples(h) -> List[Tuple]:
    p = h["pattern"].astype(np.int64)
    out = list(zip(h["record"].tolist(), (p >> 2).tolist(), h["pos"].tolist(), ((p >> 1) & 1).tolist(),
                   (p & 1).tolist(), h["mism"].tolist()))
    return sorted(out)


def oracle_hit_tuples(h) -> List[Tuple]:
    return sorted(zip(h["record"].tolist(), h["pair"].tolist(), h["pos"].tolist(), h["strand"].tolist(),
                      h["primer"].tolist(), h["mism"].tolist()))


def _gpu_site(h, i):
    x = h[i]
    return (int(x["pos"]), int((x["pattern"] >> 1) & 1), int(x["pattern"] & 1))


def _or_site(h, i):
    x = h[i]
    return (int(x["pos"]), int(x["strand"]), int(x["primer"]))


def gpu_amp_keys(out) -> List[Tuple]:
    return [(int(a["record"]), int(a["pair"]), int(a["start"]), int(a["end"]), int(a["orient"]),
             _gpu_site(out.hits, a["hit_i"]), _gpu_site(out.hits, a["hit_j"])) for a in out.amps]


def oracle_amp_keys(hits, amps) -> List[Tuple]:
    return [(int(a["record"]), int(a["pair"]), int(a["start"]), int(a["end"]), int(a["orient"]),
             _or_site(hits, a["hit_i"]), _or_site(hits, a["hit_j"])) for a in amps]


def assert_same_hits(out, ref):
    g, o = gpu_hit_tuples(out.hits), oracle_hit_tuples(ref.hits)
    assert len(g) == len(o), f"hit count {len(g)} vs oracle {len(o)}"
    for a, b in zip(g, o):
        assert a == b, f"hit {a} vs oracle {b}"


NEAR_TOL = 1e-9   # the near-threshold flag's distance (flags bit1)
# |Tm - min_tm| this close to NEAR_TOL: the two sides' Tms (equal within ~1e-13) may fall on either
# side of the flag's edge, so bit1 is not compared there
_EDGE_BAND = 1e-11


def _flag_bits(tm: float, undefined: bool, min_tm):
    """(decision, near, undefined) as the oracle's Tm implies them, and whether `near` is decidable."""
    if undefined:
        return False, False, True, True
    if min_tm is None:
        return True, False, False, True
    d = abs(tm - min_tm)
    return tm >= min_tm, d <= NEAR_TOL, False, abs(d - NEAR_TOL) > _EDGE_BAND


def assert_same_amplicons(out, ref, filtered: bool, min_tm="from_ref"):
    """Amplicons, Tm and the three flag bits, amplicon by amplicon.

    filtered: the CUDA output went through the Tm filter (compare with the oracle's kept set).
    min_tm: the threshold the CUDA run used; by default the oracle's when filtered, none otherwise
    (bit0 then means a defined Tm).  Amplicons within NEAR_TOL of the threshold must carry bit1; their
    decision (bit0, and with it membership of a filtered list) may differ from the oracle's, since it
    rests on the last digits of a double, but must agree with the CUDA path's own Tm.
    """
    if min_tm == "from_ref":
        min_tm = ref.min_tm if filtered else None
    assert not filtered or min_tm is not None
    ok_all = oracle_amp_keys(ref.hits, ref.amps)
    exp = {k: _flag_bits(float(t), bool(s), min_tm) + (float(t),)
           for k, t, s in zip(ok_all, ref.amp_tm, ref.amp_status)}
    gk = gpu_amp_keys(out)
    assert len(set(gk)) == len(gk), "duplicate amplicons"
    if filtered:
        must = {k for k, e in exp.items() if e[0] and not e[1]}
        may = {k for k, e in exp.items() if e[0] or e[1]}
        got = set(gk)
        assert must <= got, f"amplicons the oracle keeps are missing: {len(must - got)} of {len(must)}"
        assert got <= may, f"amplicons the oracle drops were kept: {len(got - may)}"
    else:
        assert sorted(gk) == sorted(ok_all), f"amplicon sets differ: {len(gk)} vs oracle {len(ok_all)}"
    worst = 0.0
    for k, a in zip(gk, out.amps):
        dec, near, undef, decidable, t = exp[k]
        flags = int(a["flags"])
        undefined = bool(flags & 4)
        assert undefined == undef, f"Tm definedness differs at {k}"
        if not undefined:
            g = float(a["tm"])
            d = abs(g - t)
            worst = max(worst, d)
            assert d <= TM_TOL, f"Tm {a['tm']!r} vs oracle {t!r} at {k}"
        else:
            assert math.isnan(float(a["tm"]))
        if decidable:
            assert bool(flags & 2) == near, f"near-threshold flag {bool(flags & 2)} vs oracle {near} at {k}"
        if near:
            assert bool(flags & 1) == (float(a["tm"]) >= min_tm), f"decision contradicts the CUDA Tm at {k}"
        else:
            assert bool(flags & 1) == dec, f"threshold decision {bool(flags & 1)} vs oracle {dec} at {k}"
        if filtered:
            assert flags & 1, f"filtered list holds an amplicon that fails the threshold at {k}"
    return worst


def assert_same_sequences(out, ref):
    """Sequences of the kept amplicons (the oracle extracts only kept ones, in order)."""
    ok = oracle_amp_keys(ref.hits, ref.amps[ref.keep])
    ref_seq = dict(zip(ok, ref.seqs))
    gk = gpu_amp_keys(out)
    assert len(gk) == len(ok)
    for m, k in enumerate(gk):
        assert out.fields(m) == ref_seq[k], f"sequence fields differ at {k}"


class Restricted:
    """The plan's output restricted to some records, renumbered as the oracle numbers a subset."""

    def __init__(self, out, records):
        records = np.asarray(records, dtype=np.int64)
        remap = {int(r): i for i, r in enumerate(records)}
        hm = np.isin(out.hits["record"], records)
        new_index = -np.ones(len(out.hits), dtype=np.int64)
        new_index[np.nonzero(hm)[0]] = np.arange(int(hm.sum()))
        self.hits = out.hits[hm].copy()
        self.hits["record"] = [remap[int(r)] for r in self.hits["record"]]
        am = np.isin(out.amps["record"], records)
        self._src = np.nonzero(am)[0]
        self.amps = out.amps[am].copy()
        self.amps["record"] = [remap[int(r)] for r in self.amps["record"]]
        self.amps["hit_i"] = new_index[self.amps["hit_i"]]
        self.amps["hit_j"] = new_index[self.amps["hit_j"]]
        assert (self.amps["hit_i"] >= 0).all() and (self.amps["hit_j"] >= 0).all()
        self._out = out

    def fields(self, m):
        return self._out.fields(int(self._src[m]))
