"""The oracle's Tm against values printed outside this repository (tests/golden/tm_published.md).

Section "Implementations" of the paper fixes the model: AHv2's Tm is that of Biopython's Tm_NN.
These pins tie the oracle to published numbers, not to a second transcription of its own tables:

* the unified free energies at 37 C (SantaLucia 1998, Table 1) fix every Watson-Crick stack, both
  per-end initiation terms and the symmetry term through dG = dH - 310.15 K dS;
* the Tm that Biopython's documentation prints for a 28-mer under the defaults fixes those terms,
  salt method 5 and the strand-concentration term together;
* the salt corrections that Biopython's documentation prints fix methods 1 and 2, the Tris/2 term
  and the Na+-equivalent of Mg2+.
"""
import os
import re

import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tm_published.md")
COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}
T37 = 310.15
DG_TOL = 0.02   # kcal/mol: the free energies were fitted on their own and printed to 0.01


def _table(name):
    text = open(GOLDEN).read()
    (sec,) = [b for b in re.split(r"\n## ", text) if b.startswith(name + " ")]
    rows = re.findall(r"^\|(.+)\|$", sec, re.M)
    return [[c.strip() for c in r.split("|")] for r in rows[2:]]   # after the header and its rule


_SCALAR = {"init GC": "init_G/C", "init AT": "init_A/T", "sym": "sym"}


def test_tables_complete():
    assert len(_table("dg37")) == 13 and len(_table("tm")) == 1 and len(_table("salt")) == 4
    # every Watson-Crick step of the unified set is listed once
    steps = {r[0] for r in _table("dg37") if r[0] not in _SCALAR}
    assert len(steps) == 10
    for s in steps:
        top, bottom = s.split("/")
        assert "".join(COMP[c] for c in top) == bottom


@pytest.mark.parametrize("term,dg", [(r[0], float(r[1])) for r in _table("dg37")])
def test_unified_free_energy(term, dg):
    if term in _SCALAR:
        got = oracle.nn_entry(oracle.NN_SCALAR, _SCALAR[term])
    else:
        got = oracle.nn_entry(oracle.NN_WC, term)
    assert got is not None, term
    dh, ds = got
    val = dh - T37 * ds / 1000.0
    assert abs(val - dg) <= DG_TOL, (term, dh, ds, val, dg)


def test_stack_lookup_uses_the_pinned_entries():
    """A fully paired duplex's sums are its pinned stacks plus its two pinned end terms, whichever
    strand a step is stored on (so the pins above reach every Watson-Crick duplex)."""
    table = {}
    for r in _table("dg37"):
        if r[0] not in _SCALAR:
            table[r[0]] = oracle.nn_entry(oracle.NN_WC, r[0])
    end = {c: oracle.nn_entry(oracle.NN_SCALAR, "init_G/C" if c in "GC" else "init_A/T") for c in "ACGT"}
    st = synth.Stream(synth.make_key(11, 77, 0))
    for _ in range(200):
        L = st.randint(2, 30)
        seq = "".join(st.choice("ACGT") for _ in range(L))
        cseq = "".join(COMP[c] for c in seq)
        dh, ds = end[seq[0]][0] + end[seq[-1]][0], end[seq[0]][1] + end[seq[-1]][1]
        for i in range(L - 1):
            fwd = seq[i:i + 2] + "/" + cseq[i:i + 2]
            rev = cseq[i + 1] + cseq[i] + "/" + seq[i + 1] + seq[i]   # the same step read from the other strand
            e = table.get(fwd) or table.get(rev)
            dh, ds = dh + e[0], ds + e[1]
        got = oracle.duplex_sums(seq, cseq)
        assert abs(got[0] - dh) < 1e-9 and abs(got[1] - ds) < 1e-9, seq


@pytest.mark.parametrize("seq,salt,na,tris,mg,tm", [(r[0], int(r[1]), float(r[2]), float(r[3]), float(r[4]),
                                                     float(r[5])) for r in _table("tm")])
def test_published_tm(seq, salt, na, tris, mg, tm):
    cseq = "".join(COMP[c] for c in seq)
    got = oracle.tm_duplex(seq, cseq, synth.TmParams(Na=na, Tris=tris, Mg=mg, saltcorr=salt))
    assert got is not None
    assert f"{got:.2f}" == f"{tm:.2f}", got


@pytest.mark.parametrize("method,na,tris,mg,corr", [(int(r[0]), float(r[1]), float(r[2]), float(r[3]),
                                                     float(r[4])) for r in _table("salt")])
@pytest.mark.parametrize("seq", ["CGTTCCAAAGATGTGGGCATGAGCTTAC", "ACGTAGCTAGGCTA"])
def test_published_salt_correction(method, na, tris, mg, corr, seq):
    """Methods 1-4 shift Tm by a constant, so Tm(method) - Tm(method 0) is the printed correction."""
    cseq = "".join(COMP[c] for c in seq)
    with_corr = oracle.tm_duplex(seq, cseq, synth.TmParams(Na=na, Tris=tris, Mg=mg, saltcorr=method))
    without = oracle.tm_duplex(seq, cseq, synth.TmParams(Na=na, Tris=tris, Mg=mg, saltcorr=0))
    assert f"{with_corr - without:.2f}" == f"{corr:.2f}", with_corr - without
