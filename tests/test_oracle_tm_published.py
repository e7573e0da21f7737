"""The oracle's Tm against values printed outside this repository (tests/golden/tm_published.md).

Section "Implementations" of the paper fixes the model: AHv2's Tm is that of Biopython's Tm_NN.
These pins tie the oracle to published numbers, not to a second transcription of its own tables:

* the unified free energies at 37 C (SantaLucia 1998, Table 1) fix every Watson-Crick stack, both
  per-end initiation terms and the symmetry term through dG = dH - 310.15 K dS;
* the Tm that Biopython's documentation prints for a 28-mer under the defaults fixes those terms,
  salt method 5 and the strand-concentration term together;
* the salt corrections that Biopython's documentation prints fix methods 1 and 2, the Tris/2 term
  and the Na+-equivalent of Mg2+;
* the free energies printed beside the other Watson-Crick sets (Breslauer 1986, Sugimoto 1996,
  SantaLucia & Hicks 2004, Freier 1986, Sugimoto 1995) fix each set's stacks and scalar terms.
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


# ---------------------------------------------------------------------------------------- other sets
_SET_STACKS = {1: 10, 2: 10, 4: 10, 5: 10, 8: 16}   # stacks each set stores (8: RNA/DNA, not symmetric)


def test_sets_complete():
    rows = _table("sets")
    for st, n in _SET_STACKS.items():
        steps = {r[1] for r in rows if int(r[0]) == st and "/" in r[1] and not r[1].startswith("init")}
        assert len(steps) == n, (st, len(steps))
        for s in steps:
            top, bottom = s.split("/")
            assert "".join(COMP[c] for c in top) == bottom
            assert oracle.nn_entry(oracle.NN_WC, s, st) is not None, (st, s)


@pytest.mark.parametrize("row", _table("sets"), ids=lambda r: f"set{r[0]}-{r[1]}")
def test_set_free_energy(row):
    st, term, T, dg, tol = int(row[0]), row[1], float(row[2]), float(row[3]), float(row[4])
    wc = "/" in term and not term.startswith("init")
    got = oracle.nn_entry(oracle.NN_WC if wc else oracle.NN_SCALAR, term, st)
    assert got is not None, (st, term)
    val = got[0] - T * got[1] / 1000.0
    assert abs(val - dg) <= tol, (st, term, got, val, dg)


@pytest.mark.parametrize("st", sorted(_SET_STACKS))
def test_set_sums_use_the_pinned_entries(st):
    """A fully paired duplex's sums under set `st` are its pinned stacks plus the set's pinned
    initiation terms: every duplex, per terminal pair, G/C present or absent, 5' T and 3' A.  The
    shared mismatch tables play no part, so this reaches every entry of the set's stack table."""
    stacks = {r[1]: oracle.nn_entry(oracle.NN_WC, r[1], st) for r in _table("sets")
              if int(r[0]) == st and "/" in r[1] and not r[1].startswith("init")}
    sc = {k: oracle.nn_entry(oracle.NN_SCALAR, k, st)
          for k in ("init", "init_A/T", "init_G/C", "init_oneG/C", "init_allA/T", "init_5T/A")}
    st_rng = synth.Stream(synth.make_key(st, 77, 2))
    for _ in range(200):
        L = st_rng.randint(2, 30)
        seq = "".join(st_rng.choice(st_rng.choice(["ACGT", "AT"])) for _ in range(L))
        cseq = "".join(COMP[c] for c in seq)
        terms = [sc["init"], sc["init_oneG/C"] if any(c in "GC" for c in seq) else sc["init_allA/T"]]
        terms += [sc["init_G/C"] if c in "GC" else sc["init_A/T"] for c in (seq[0], seq[-1])]
        terms += [sc["init_5T/A"]] * ((seq[0] == "T") + (seq[-1] == "A"))
        for i in range(L - 1):
            fwd = seq[i:i + 2] + "/" + cseq[i:i + 2]
            rev = cseq[i + 1] + cseq[i] + "/" + seq[i + 1] + seq[i]
            terms.append(stacks.get(fwd) or stacks.get(rev))
        dh, ds = sum(t[0] for t in terms), sum(t[1] for t in terms)
        got = oracle.duplex_sums(seq, cseq, st)
        assert abs(got[0] - dh) < 1e-9 and abs(got[1] - ds) < 1e-9, (st, seq)


def test_unbuilt_sets_are_refused():
    """RNA_NN2 and RNA_NN3 (6, 7) are not built: no entries, no sums."""
    for st in (6, 7, 9, -1):
        assert oracle.nn_entry(oracle.NN_WC, "AA/TT", st) is None
        assert oracle.duplex_sums("ACGT", "TGCA", st) is None
