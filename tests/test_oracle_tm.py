"""Pins for the oracle's nearest-neighbour Tm (Section "Implementations": AHv2's C Tm_NN; Section
"Primer degeneracy": Tm over primer variants).

* hand-worked sums (tests/golden/tm_worked.md) pin which terms apply: terminal mismatches, the
  reversed-step lookup, initiation on the written strand's ends, tandem G.T steps, undefined steps;
* a fully Watson-Crick duplex reduces to the closed form built from a second, independent entry of
  the stack parameters (a 16-dinucleotide matrix), which also double-checks the oracle's table;
* reading a duplex from the other strand leaves Tm unchanged (no terminal mismatch);
* the salt correction of method 5 vanishes at 1 M monovalent salt and raises Tm with [Na+];
* every single mismatch next to a Watson-Crick pair has a parameter;
* the degenerate-primer Tm is the maximum over the brute-force list of concrete variants.
"""
import math
import os
import re

import pytest

import oracle
import synth
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tm_worked.md")
COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def _worked():
    text = open(GOLDEN).read()
    out = []
    for block in re.split(r"\n## ", text)[1:]:
        head = block.splitlines()[0]
        m = re.match(r"(\S+) seq=(\S+) cseq=(\S+)", head)
        rows = re.findall(r"^\| ([^|]+?) \| [^|]*\| (-?\d+\.\d+) \| (-?\d+\.\d+) \|$", block, re.M)
        out.append((m.group(1), m.group(2), m.group(3), [(r[0], float(r[1]), float(r[2])) for r in rows]))
    return out


@pytest.mark.parametrize("name,seq,cseq,rows", _worked())
def test_hand_worked_sums(name, seq, cseq, rows):
    got = oracle.duplex_sums(seq, cseq)
    if name == "undefined":
        assert got is None
        return
    terms = [r for r in rows if r[0] != "total"]
    (total,) = [r for r in rows if r[0] == "total"]
    assert abs(sum(t[1] for t in terms) - total[1]) < 1e-9
    assert abs(sum(t[2] for t in terms) - total[2]) < 1e-9
    assert got is not None
    assert abs(got[0] - total[1]) < 1e-9 and abs(got[1] - total[2]) < 1e-9


# Second entry of the Watson-Crick stacks (Allawi & SantaLucia 1997), indexed by the top-strand
# dinucleotide 5'->3' of a fully paired duplex: (dH kcal/mol, dS cal/(K mol)).
DINUC = {
    "AA": (-7.9, -22.2), "AC": (-8.4, -22.4), "AG": (-7.8, -21.0), "AT": (-7.2, -20.4),
    "CA": (-8.5, -22.7), "CC": (-8.0, -19.9), "CG": (-10.6, -27.2), "CT": (-7.8, -21.0),
    "GA": (-8.2, -22.2), "GC": (-9.8, -24.4), "GG": (-8.0, -19.9), "GT": (-8.4, -22.4),
    "TA": (-7.2, -21.3), "TC": (-8.2, -22.2), "TG": (-8.5, -22.7), "TT": (-7.9, -22.2),
}
END = {"A": (2.3, 4.1), "T": (2.3, 4.1), "G": (0.1, -2.8), "C": (0.1, -2.8)}


def closed_form_tm(seq, Na=50.0, c1=25.0, c2=25.0):
    dh = sum(DINUC[seq[i:i + 2]][0] for i in range(len(seq) - 1)) + END[seq[0]][0] + END[seq[-1]][0]
    ds = sum(DINUC[seq[i:i + 2]][1] for i in range(len(seq) - 1)) + END[seq[0]][1] + END[seq[-1]][1]
    ds += 0.368 * (len(seq) - 1) * math.log(Na / 1000.0)
    return 1000.0 * dh / (ds + 1.987 * math.log((c1 - c2 / 2.0) * 1e-9)) - 273.15


@pytest.mark.parametrize("seed", range(20))
def test_watson_crick_closed_form(seed):
    st = synth.Stream(synth.make_key(seed, 77, 0))
    seq = "".join(st.choice("ACGT") for _ in range(st.randint(8, 30)))
    cseq = "".join(COMP[c] for c in seq)
    Na = [50.0, 10.0, 200.0][seed % 3]
    tm = oracle.tm_duplex(seq, cseq, synth.TmParams(Na=Na))
    assert abs(tm - closed_form_tm(seq, Na=Na)) < 1e-9


def test_duplex_read_from_other_strand():
    st = synth.Stream(synth.make_key(5, 78, 0))
    n = 0
    for _ in range(300):
        L = st.randint(10, 26)
        seq = "".join(st.choice("ACGT") for _ in range(L))
        cseq = list(COMP[c] for c in seq)
        # up to two isolated internal mismatches, ends stay paired
        for p in st.sample(L - 4, 2)[: st.randint(0, 2)]:
            q = p + 2
            cseq[q] = st.choice([b for b in "ACGT" if b != COMP[seq[q]]])
        cseq = "".join(cseq)
        t1 = oracle.tm_duplex(seq, cseq, synth.TmParams())
        t2 = oracle.tm_duplex(cseq[::-1], seq[::-1], synth.TmParams())
        assert (t1 is None) == (t2 is None)
        if t1 is not None:
            assert abs(t1 - t2) < 1e-9
            n += 1
    assert n > 100


def test_every_single_mismatch_step_has_a_parameter():
    wc = [("A", "T"), ("C", "G"), ("G", "C"), ("T", "A")]
    mism = [(x, y) for x in "ACGT" for y in "ACGT" if COMP[x] != y]
    for a, ca in wc:
        for x, y in mism:
            for left in (True, False):
                # G.C clamps on both sides keep the mismatch internal
                s = "GC" + (a + x if left else x + a) + "GC"
                c = "CG" + (ca + y if left else y + ca) + "CG"
                assert oracle.duplex_sums(s, c) is not None, (s, c)
                # as a terminal mismatch next to a Watson-Crick pair (right end of the duplex)
                s2, c2 = "GCGC" + a + x, "CGCG" + ca + y
                ref = oracle.duplex_sums(s2[:-1], c2[:-1])
                got = oracle.duplex_sums(s2, c2)
                assert got is not None and ref is not None


def test_salt_method5():
    seq = "AGCTTGACCGTAGGCATTA"
    cseq = "".join(COMP[c] for c in seq)
    at_1M = oracle.tm_duplex(seq, cseq, synth.TmParams(Na=1000.0))
    none = oracle.tm_duplex(seq, cseq, synth.TmParams(saltcorr=0))
    assert abs(at_1M - none) < 1e-9
    ts = [oracle.tm_duplex(seq, cseq, synth.TmParams(Na=na)) for na in (5, 20, 50, 100, 300)]
    assert all(a < b for a, b in zip(ts, ts[1:]))


@pytest.mark.parametrize("seq", ["AGCTTGACCGTAGGCATTA", "GCGCGGCCGCATGC", "ATATTAAATTTATATAATAT"])
@pytest.mark.parametrize("na", [10.0, 50.0, 200.0])
def test_salt_method7_without_magnesium_is_method6(seq, na):
    """Owczarzy et al. 2008 reduces to Owczarzy et al. 2004 (method 6) when no Mg2+ is present: the
    Mg2+ / monovalent ratio is 0, below the 0.22 bound where monovalent ions dominate."""
    cseq = "".join(COMP[c] for c in seq)
    m6 = oracle.tm_duplex(seq, cseq, synth.TmParams(Na=na, saltcorr=6))
    m7 = oracle.tm_duplex(seq, cseq, synth.TmParams(Na=na, saltcorr=7))
    assert m6 is not None and abs(m6 - m7) < 1e-12


@pytest.mark.parametrize("seq", ["AGCTTGACCGTAGGCATTA", "GCGCGGCCGCATGC"])
def test_salt_method7_magnesium_dominated_ignores_monovalent(seq):
    """At sqrt([Mg2+]) / [Mon+] >= 6 (Owczarzy et al. 2008) the correction depends on Mg2+ alone:
    10 mM Mg2+ (sqrt 0.1 M^1/2) with 0 to 16 mM monovalent ions gives one Tm; 20 mM Na+ (ratio
    5) falls in the mixed regime and differs."""
    cseq = "".join(COMP[c] for c in seq)
    ts = [oracle.tm_duplex(seq, cseq, synth.TmParams(Na=na, Mg=10.0, saltcorr=7)) for na in (0.0, 5.0, 10.0, 16.0)]
    assert ts[0] is not None and max(ts) - min(ts) < 1e-12
    mixed = oracle.tm_duplex(seq, cseq, synth.TmParams(Na=20.0, Mg=10.0, saltcorr=7))
    assert abs(mixed - ts[0]) > 1e-6


def test_salt_method7_tm_rises_with_magnesium():
    """Tm of a 19-mer rises with Mg2+ over the PCR range 0.5-10 mM at 50 mM Na+ (Owczarzy et al. 2008)."""
    seq = "AGCTTGACCGTAGGCATTA"
    cseq = "".join(COMP[c] for c in seq)
    ts = [oracle.tm_duplex(seq, cseq, synth.TmParams(Na=50.0, Mg=mg, saltcorr=7)) for mg in (0.5, 1.0, 2.0, 5.0, 10.0)]
    assert all(a < b for a, b in zip(ts, ts[1:])), ts
    # and without any cation the method is undefined
    assert oracle.tm_duplex(seq, cseq, synth.TmParams(Na=0.0, Mg=0.0, saltcorr=7)) is None


@pytest.mark.parametrize("mg,dntp", [(1.5, 0.8), (3.0, 0.2), (2.0, 2.0), (0.5, 4.0), (10.0, 1.0)])
def test_free_magnesium_satisfies_mass_action(mg, dntp):
    """Free Mg2+ beside dNTPs (Ka = 3e4 per M, one to one): Ka [Mg]free [dNTP]free = [Mg.dNTP], with
    both free amounts non-negative and the bound amount at most the smaller total."""
    x = oracle.free_mg(mg, dntp) * 1e-3
    bound = mg * 1e-3 - x
    dfree = dntp * 1e-3 - bound
    assert 0.0 < x <= mg * 1e-3 and 0.0 <= bound <= min(mg, dntp) * 1e-3 + 1e-15 and dfree >= -1e-15
    assert abs(3e4 * x * dfree - bound) <= 1e-9 * max(bound, 1e-12)
    assert oracle.free_mg(mg, 0.0) == mg


@pytest.mark.parametrize("seq", ["GCGCAATTGCGC", "ACGTACGT", "AGCTTAAGCT"])
def test_self_complementary_duplex(seq):
    """A self-complementary duplex (selfcomp) takes C = c1 and the symmetry entropy: its Tm equals the
    ordinary Tm at strand concentration c1 exp(dS_sym / R), c2 = 0, with dS_sym = -1.4 cal/(K mol)."""
    cseq = "".join(COMP[c] for c in seq)
    assert "".join(COMP[c] for c in reversed(seq)) == seq
    for salt in (0, 5, 6):
        sc = oracle.tm_duplex(seq, cseq, synth.TmParams(dnac1=250.0, dnac2=0.0, saltcorr=salt, selfcomp=1))
        eq = oracle.tm_duplex(seq, cseq, synth.TmParams(dnac1=250.0 * math.exp(-1.4 / 1.987), dnac2=0.0,
                                                        saltcorr=salt))
        assert abs(sc - eq) < 1e-9, (salt, sc, eq)


def test_concentration_term():
    seq = "AGCTTGACCGTAGGCATTA"
    cseq = "".join(COMP[c] for c in seq)
    # C = c1 - c2/2: 25/25 nM equals 12.5/0 nM
    a = oracle.tm_duplex(seq, cseq, synth.TmParams(dnac1=25, dnac2=25))
    b = oracle.tm_duplex(seq, cseq, synth.TmParams(dnac1=12.5, dnac2=0))
    assert abs(a - b) < 1e-12
    assert oracle.tm_duplex(seq, cseq, synth.TmParams(dnac1=250, dnac2=250)) > a


def _qualifying(primer, site, k, clamp):
    """Brute force: concrete variants of `primer` with at most k mismatches to `site` and none in the
    last `clamp` positions."""
    L = len(primer)
    out = []
    for v in brute.variants(primer):
        diff = [i for i in range(L) if v[i] != site[i]]
        if len(diff) <= k and all(i < L - clamp for i in diff):
            out.append(v)
    return out


@pytest.mark.parametrize("primer,site,k,clamp", [
    ("ACGTRYACGTAGG", "ACGTACACGTAGG", 13, 0),
    ("NACGTAGCWAGT", "TACGTAGCAAGT", 12, 0),
    ("GGCATKMSACGTTA", "GGCATGCCACGTTA", 2, 3),
    ("BDHVACGGT", "CATGACGGT", 1, 2),
    ("ACGGTTNNAC", "ACGGTTAGAC", 0, 0),
    ("ACGGTTNNAC", "ACGGTTAGAC", 2, 4),
    ("ANCCTRGTCVYHTBN", "ACCCTTGGCACGTTC", 3, 2),
])
def test_degenerate_tm_is_max_over_qualifying_variants(primer, site, k, clamp):
    """Reading R14: the maximum of the duplex Tm over the variants that match the site within k
    mismatches and the exact clamp, checked against a brute-force filter of every variant."""
    cseq = "".join(COMP[c] for c in site)
    vals = [oracle.tm_duplex(v, cseq, synth.TmParams()) for v in _qualifying(primer, site, k, clamp)]
    vals = [v for v in vals if v is not None]
    got = oracle.tm_site(primer, site, synth.TmParams(), k=k, clamp=clamp)
    if not vals:
        assert got is None
    else:
        assert got is not None and abs(got - max(vals)) < 1e-12


def test_site_tm_concrete_primer():
    """A primer without degenerate codes has one variant: its own duplex Tm when the site is within k
    mismatches and the clamp is exact, else undefined."""
    primer = "AGCTTGACCGTAGGCA"
    site = "AGCTTGACCATAGGCA"   # one mismatch, 6 positions from the 3' end
    cseq = "".join(COMP[c] for c in site)
    t = oracle.tm_duplex(primer, cseq, synth.TmParams())
    assert t is not None
    assert oracle.tm_site(primer, site, synth.TmParams(), k=1, clamp=6) == t
    assert oracle.tm_site(primer, site, synth.TmParams(), k=0, clamp=0) is None
    assert oracle.tm_site(primer, site, synth.TmParams(), k=1, clamp=7) is None


def test_site_tm_excludes_far_variants():
    """A variant that differs from the site at many positions can reach a larger Biopython value
    (here the entropy sum comes near -R ln C); it does not count unless it matches the site."""
    primer, site = "ANCCTRGTCVYHTBN", "ACCCTTGGCACGTTC"
    prm = synth.TmParams(Na=10.0, saltcorr=4)
    every = oracle.tm_site(primer, site, prm)
    near = oracle.tm_site(primer, site, prm, k=3, clamp=2)
    assert every is not None and near is not None
    assert every > 200.0 and near < 100.0
    cseq = "".join(COMP[c] for c in site)
    vals = [oracle.tm_duplex(v, cseq, prm) for v in _qualifying(primer, site, 3, 2)]
    assert abs(near - max(v for v in vals if v is not None)) < 1e-12




@pytest.mark.parametrize("variants", [0, 1])
def test_hit_tm_follows_the_variant_option(variants):
    """Per-hit Tm: every variant by default, the site-matching ones (the pair's k, the clamp) with
    variants = 1; checked hit by hit against the site-level function on the site's own bases."""
    import dataclasses

    wl = synth.random_small(5, n_records=20, len_lo=200, len_hi=800, n_pairs=2, plen_lo=8, plen_hi=12, n_deg=4,
                            k_max=3, clamp=2, plant=3)
    wl.tm = dataclasses.replace(wl.tm, variants=variants)
    hits = oracle.scan(wl)
    assert len(hits) > 5
    tm, st = oracle.tm_hits(wl, hits)
    for h, t, s in zip(hits, tm, st):
        P = (wl.fwd if h["primer"] == 0 else wl.rev)[h["pair"]]
        L = len(P)
        g = wl.seq[wl.offsets[h["record"]]:wl.offsets[h["record"] + 1]].tobytes().decode().upper()
        site = g[h["pos"]:h["pos"] + L]
        if h["strand"] == 1:
            site = "".join(COMP[c] for c in reversed(site))
        k, c = (wl.k[h["pair"]], wl.clamp) if variants else (None, 0)
        r = oracle.tm_site(P, site, wl.tm, k=k, clamp=c)
        if r is None:
            assert s == 1
        else:
            assert s == 0 and t == r
