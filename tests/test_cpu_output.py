"""FASTA output (ah_amplicons_fasta, host code of the library, no GPU) against the reference
formatter written from Supplementary "Headers and outputs", on the oracle's own amplicons and
sequences: every orientation, barcodes on and off, sources present and absent, undefined Tm."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def ah():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2511_00170_gb300 import ah as mod

    return mod


def _inputs(seed):
    wl = synth.random_small(seed, n_records=5, len_lo=300, len_hi=5000, n_pairs=2, plant=3, fb=6, rb=4, trim=bool(seed % 2))
    wl.orient_mask = 15
    ref = oracle.run(wl)
    kept = np.nonzero(ref.keep)[0]
    amps = ref.amps[kept]
    tms = ref.amp_tm[kept].astype(np.float64)
    tms[ref.amp_status[kept] != 0] = np.nan
    fields = [tuple(x if isinstance(x, bytes) else x.encode() for x in f) for f in ref.seqs]
    return wl, amps, tms, fields


@pytest.mark.parametrize("seed", [3, 8, 13, 21])
@pytest.mark.parametrize("barcodes,with_sources", [(True, True), (False, False)])
def test_amplicon_fasta_matches_reference(ah, seed, barcodes, with_sources):
    wl, amps, tms, fields = _inputs(seed)
    assert len(amps) > 0 and len(set(int(o) for o in amps["orient"])) >= 2
    abi = np.zeros(len(amps), dtype=ah.AMP_DTYPE)
    for k in ("record", "start", "end", "orient", "hit_i", "hit_j"):
        abi[k] = amps[k]
    abi["pair"] = amps["pair"]
    abi["tm"] = tms
    arena = b"".join(b"".join(f) for f in fields)
    off = np.zeros(5 * len(fields) + 1, dtype=np.uint64)
    pos = 0
    for m, f in enumerate(fields):
        for k in range(5):
            off[5 * m + k] = pos
            pos += len(f[k])
    off[-1] = pos
    names = ["rec%d Escherichia coli strain %d" % (r, r) for r in range(wl.n_records)]
    sources = ["GCF_%06d.fa" % (1000 + r) for r in range(wl.n_records)] if with_sources else None
    got = ah.ah_amplicons_fasta(abi, arena, off, names, sources, barcodes)
    recs = [(int(a["record"]), int(a["start"]), int(a["end"]), int(a["orient"]), float(t), f)
            for a, t, f in zip(amps, tms, fields)]
    want = oracle.amplicon_fasta(recs, names, sources, barcodes)
    assert got == want
    assert got.count(b"\n>") + 1 == len(amps)


def test_amplicon_fasta_refuses_bad_record(ah):
    abi = np.zeros(1, dtype=ah.AMP_DTYPE)
    abi["record"] = 3
    with pytest.raises(ah.AhError):
        ah.ah_amplicons_fasta(abi, b"ACGT", np.array([0, 4, 4, 4, 4, 4], dtype=np.uint64), ["r0"], None, False)


def test_amplicon_fasta_paper_example_shape(ah):
    """The header of the paper's example (Supplementary "Headers and outputs"): id, source,
    coordinates, Tm to two decimals, orientation, primer sites, barcodes; and NA for an undefined Tm."""
    abi = np.zeros(2, dtype=ah.AMP_DTYPE)
    abi["record"] = [0, 0]
    abi["start"] = [12344, 99]
    abi["end"] = [13567, 150]
    abi["orient"] = [0, 1]
    abi["tm"] = [60.4249, np.nan]
    fields = [b"ACGTTT", b"ACGT", b"TGCA", b"AAC", b"GGT", b"CC", b"", b"", b"TTA", b"CAG"]
    off = np.cumsum([0] + [len(f) for f in fields]).astype(np.uint64)
    got = ah.ah_amplicons_fasta(abi, b"".join(fields), off, ["seqid some text"], ["GCF_XXXX.fa"], True)
    assert got == (b">seqid.source=GCF_XXXX.fa.coordinates=12345-13567.Tm=60.42.orientation=FR"
                   b".fprimer=AAC.rprimer=GGT.fb=ACGT.rb=TGCA\nACGTTT\n"
                   b">seqid.source=GCF_XXXX.fa.coordinates=100-150.Tm=NA.orientation=RF"
                   b".fprimer=CAG.rprimer=TTA.fb=.rb=\nCC\n")
    recs = [(0, 12344, 13567, 0, 60.4249, tuple(fields[0:5])), (0, 99, 150, 1, float("nan"), tuple(fields[5:10]))]
    assert oracle.amplicon_fasta(recs, ["seqid some text"], ["GCF_XXXX.fa"], True) == got


@pytest.mark.parametrize("seed", [3, 8])
def test_amplicon_fastq_matches_reference(ah, seed):
    """FASTQ output: the FASTA header with '@', the sequence, '+' and the qualities of field 0."""
    wl, amps, tms, fields = _inputs(seed)
    abi = np.zeros(len(amps), dtype=ah.AMP_DTYPE)
    for k in ("record", "start", "end", "orient", "hit_i", "hit_j"):
        abi[k] = amps[k]
    abi["tm"] = tms
    arena = b"".join(b"".join(f) for f in fields)
    off = np.cumsum([0] + [len(x) for f in fields for x in f]).astype(np.uint64)
    # qualities: any printable bytes of the amplicon's length, at field 0's offsets
    rng = np.random.default_rng(seed)
    q = [bytes(rng.integers(33, 74, len(f[0]), dtype=np.uint8)) for f in fields]
    qarena = bytearray(len(arena))
    for m, f in enumerate(fields):
        qarena[int(off[5 * m]):int(off[5 * m]) + len(f[0])] = q[m]
    names = ["rec%d x" % r for r in range(wl.n_records)]
    got = ah.ah_amplicons_fastq(abi, arena, bytes(qarena), off, names, None, True)
    recs = [(int(a["record"]), int(a["start"]), int(a["end"]), int(a["orient"]), float(t), f, qq)
            for a, t, f, qq in zip(amps, tms, fields, q)]
    assert got == oracle.amplicon_fastq(recs, names, None, True)
    assert got.count(b"\n+\n") == len(amps)


def test_amplicon_fasta_into_caller_buffer(ah):
    """With `out`, the text goes into the caller's array and its length comes back; an array too
    small for it is refused before anything is written."""
    wl, amps, tms, fields = _inputs(8)
    abi = np.zeros(len(amps), dtype=ah.AMP_DTYPE)
    for k in ("record", "start", "end", "orient", "hit_i", "hit_j"):
        abi[k] = amps[k]
    abi["tm"] = tms
    arena = b"".join(b"".join(f) for f in fields)
    off = np.cumsum([0] + [len(x) for f in fields for x in f]).astype(np.uint64)
    names = ["rec%d x" % r for r in range(wl.n_records)]
    want = ah.ah_amplicons_fasta(abi, arena, off, names, None, True)
    buf = np.full(len(want) + 10, 0xAB, dtype=np.uint8)
    n = ah.ah_amplicons_fasta(abi, arena, off, names, None, True, out=buf)
    assert n == len(want) and buf[:n].tobytes() == want and np.all(buf[n:] == 0xAB)
    with pytest.raises(ValueError):
        ah.ah_amplicons_fasta(abi, arena, off, names, None, True, out=np.zeros(len(want) - 1, dtype=np.uint8))
