"""Every nearest-neighbour set of Tm_NN against the oracle, through the C ABI (needs a GPU).

Section "Implementations": the Tm is Biopython's Tm_NN with any parameter combination.  Each Watson-
Crick set (Breslauer 1986, Sugimoto 1996, the default Allawi & SantaLucia 1997, SantaLucia & Hicks
2004, Freier 1986 for RNA, Sugimoto 1995 for RNA/DNA) is checked on duplexes with mismatches, on
degenerate sites by every site kernel (the generated and the built-in chain, the lane groups of the
site-matching reading, the enumeration), and through the whole path.  Breslauer's initiation
depends on whether a duplex holds G or C at all, so A/T-only primers and duplexes are included.
"""
import math

import pytest

import oracle
import synth
from tests import compare
from tests.test_gpu_tm_kernels import _planted_case, _step

pytestmark = pytest.mark.gpu

SETS = [1, 2, 3, 4, 5, 8]
COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


@pytest.fixture(scope="module")
def engine():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2511_00170_gb300.pipeline import Engine

    e = Engine(0)
    yield e
    e.close()


def _duplexes(seed, n):
    st = synth.Stream(synth.make_key(seed, 903, 0))
    seqs, cseqs = [], []
    for _ in range(n):
        L = st.randint(2, 32)
        s = "".join(st.choice(st.choice(["ACGT", "ACGT", "AT"])) for _ in range(L))
        c = [COMP[x] for x in s]
        for _ in range(st.randint(0, 4)):
            p = st.randint(0, L - 1)
            c[p] = st.choice([b for b in "ACGT" if b != COMP[s[p]]])
        seqs.append(s)
        cseqs.append("".join(c))
    return seqs, cseqs


@pytest.mark.parametrize("nn", SETS)
def test_duplexes(engine, nn):
    from paper_2511_00170_gb300 import ah

    seqs, cseqs = _duplexes(nn, 4000)
    for case in (dict(Na=50.0, saltcorr=5), dict(Na=20.0, saltcorr=1), dict(Na=50.0, Mg=2.0, saltcorr=7),
                 dict(Na=50.0, saltcorr=5, selfcomp=1, dnac1=250.0)):
        got = ah.ah_tm_duplexes(engine.ctx, seqs, cseqs, ah.tm_params(nn_table=nn, **case))
        tmp = synth.TmParams(nn_table=nn, **case)
        for s, c, g in zip(seqs, cseqs, got):
            r = oracle.tm_duplex(s, c, tmp)
            if r is None:
                assert math.isnan(g), (nn, case, s, c)
            else:
                assert abs(g - r) <= compare.TM_TOL, (nn, case, s, c, g, r)


def _sites(seed, n, codes):
    st = synth.Stream(synth.make_key(seed, 904, 1))
    prims, sites, ks, clamps = [], [], [], []
    for i in range(n):
        L = st.randint(12, 20)
        # every other primer without any C or G fixed in it: its variants may hold none
        if i % 2:
            p = "".join(st.choice("WNRYKMDH") if st.unit() < 0.3 else st.choice("AT") for _ in range(L))
        else:
            p = synth.random_primer(st, L, st.randint(3, 8), 0, codes)
        v = synth.concrete_variant(st, p)
        sites.append(synth.substitute(st, v, st.randint(0, 3)))
        prims.append(p)
        ks.append(st.randint(0, 4))
        clamps.append(st.randint(0, 3))
    return prims, sites, ks, clamps


@pytest.mark.parametrize("nn", [1, 4, 5, 8])
def test_degenerate_sites(engine, nn):
    """The site-matching reading (lane groups, or the per-thread chain and enumeration) and the
    every-variant reading, for primers with and without a fixed C or G."""
    from paper_2511_00170_gb300 import ah

    prims, sites, ks, clamps = _sites(nn, 30, "RYSWKMBDHVN")
    for method in (5, 4):
        prm = ah.tm_params(Na=10.0 if method == 4 else 50.0, saltcorr=method, nn_table=nn)
        tmp = synth.TmParams(Na=10.0 if method == 4 else 50.0, saltcorr=method, nn_table=nn)
        for k, cl in ((ks, clamps), (None, None)):
            got = ah.ah_tm_sites(engine.ctx, prims, sites, prm, k=k, clamp=cl)
            for i, (p, s, g) in enumerate(zip(prims, sites, got)):
                r = oracle.tm_site(p, s, tmp, k=None if k is None else k[i], clamp=0 if cl is None else cl[i])
                if r is None:
                    assert math.isnan(g), (nn, p, s)
                else:
                    assert abs(g - r) <= compare.TM_TOL, (nn, p, s, g, r)


@pytest.mark.parametrize("nn", SETS)
def test_whole_path_both_site_kernels(engine, nn):
    """Planted sites of a degenerate pair through the whole path, with the generated and the built-in
    site kernel; set 1 also with an A/T-only pair (its chain gives way to enumeration)."""
    pairs = [("NNRYTGACCGTAGSAN", "NAGYCGATWKSGNACT", 3)]
    if nn == 1:
        pairs.append(("WATWRATTWAYTAAWT", "TWAWTRATWATAWATA", 2))
    for j, (fwd, rev, k) in enumerate(pairs):
        wl = _planted_case(70 + 10 * nn + j, fwd, rev, k)
        wl.tm.nn_table = nn
        ref = oracle.run(wl, with_seqs=False)
        assert len(ref.amps) > 0
        for mode in (0, 1):
            out, st = _step(engine, wl, mode)
            assert st["tm_generated" if mode == 0 else "tm_builtin"] == 1, (nn, mode, st)
            compare.assert_same_hits(out, ref)
            compare.assert_same_amplicons(out, ref, filtered=False)


def test_unbuilt_sets_refused(engine):
    from paper_2511_00170_gb300 import ah

    for nn in (6, 7, 9, -1):
        with pytest.raises(ah.AhError) as e:
            ah.ah_tm_duplexes(engine.ctx, ["ACGT"], ["TGCA"], ah.tm_params(nn_table=nn))
        assert e.value.status == ah.AH_EINVAL
