"""FASTA input parsed and packed on the device (ah_fasta_pack) against the oracle's line-by-line
parser: record names, and packed planes and invalid words identical to packing the oracle's record
sequences (needs a GPU)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ah_ctx():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2511_00170_gb300 import ah

    ctx = ah.ah_ctx_create(0)
    yield ah, ctx
    ah.ah_ctx_destroy(ctx)


def _random_fasta(seed: int, n_records: int, crlf: bool, junk: bool) -> bytes:
    st = synth.Stream(synth.make_key(seed, 4321, 0))
    nl = b"\r\n" if crlf else b"\n"
    out = bytearray()
    if junk:
        out += b"; a comment line before the first record" + nl + b"ACGT" + nl
    for r in range(n_records):
        name_len = st.choice([5, 30, 200, 5000])   # 5000: a header longer than a 4 KiB tile
        name = "rec%d " % r + "".join(st.choice("abcXYZ0123 _|=.") for _ in range(name_len))
        out += b">" + name.encode() + nl
        L = st.choice([0, 1, 50, 999, 10000, 70000])
        seq = "".join(st.choice("ACGTACGTACGTacgtNnRY") for _ in range(L))
        width = st.choice([60, 61, 80, 10 ** 9])   # 10**9: one line per record
        for i in range(0, L, width):
            line = seq[i:i + width]
            if st.randint(0, 20) == 0:
                line = line[: len(line) // 2] + " \t" + line[len(line) // 2:]
            out += line.encode() + nl
        if st.randint(0, 5) == 0:
            out += nl   # an empty line
    if out.endswith(nl) and st.randint(0, 1):
        out = out[: -len(nl)]   # no final line break
    return bytes(out)


def _batch_bytes(ah, batch):
    planes, groups, words = ah.ah_batch_export(batch)
    v = ah.ah_batch_view_get(batch)
    return planes.tobytes(), groups.tobytes(), words.tobytes(), v["n_records"], v["n_bases"]


@pytest.mark.parametrize("seed,n_records,crlf,junk,on_device",
                         [(1, 1, False, False, False), (2, 7, False, True, False), (3, 40, True, False, False),
                          (4, 25, False, False, True), (5, 60, True, True, True), (6, 3, False, False, True)])
def test_fasta_pack_matches_oracle(ah_ctx, seed, n_records, crlf, junk, on_device):
    import torch

    ah, ctx = ah_ctx
    text = _random_fasta(seed, n_records, crlf, junk)
    names, seqs = oracle.parse_fasta(text)
    assert len(names) == n_records
    if on_device:
        d = torch.frombuffer(bytearray(text), dtype=torch.uint8).cuda()
        batch, got_names = ah.ah_fasta_pack(ctx, d.data_ptr(), n_bytes=len(text))
    else:
        batch, got_names = ah.ah_fasta_pack(ctx, text)
    lens = np.array([len(s) for s in seqs], dtype=np.uint64)
    ref = ah.ah_pack_batch(ctx, np.frombuffer(b"".join(seqs) or b"\0", dtype=np.uint8),
                           np.concatenate([[0], np.cumsum(lens)]).astype(np.int64))
    try:
        assert got_names == names
        assert _batch_bytes(ah, batch) == _batch_bytes(ah, ref)
    finally:
        ah.ah_batch_free(batch)
        ah.ah_batch_free(ref)


def test_fasta_pack_into_existing_batch(ah_ctx):
    """Packing FASTA into an existing batch of the same record lengths gives the same bases as a new
    batch; other lengths are refused."""
    ah, ctx = ah_ctx
    text = _random_fasta(7, 12, False, False)
    names, seqs = oracle.parse_fasta(text)
    fresh, _ = ah.ah_fasta_pack(ctx, text)
    into = ah.ah_batch_create(ctx, np.array([len(s) for s in seqs], dtype=np.uint64))
    wrong = ah.ah_batch_create(ctx, np.array([len(s) + 1 for s in seqs], dtype=np.uint64))
    try:
        assert ah.ah_fasta_pack_into(ctx, text, into, names=True) == names
        assert _batch_bytes(ah, into) == _batch_bytes(ah, fresh)
        with pytest.raises(ah.AhError) as e:
            ah.ah_fasta_pack_into(ctx, text, wrong)
        assert e.value.status == ah.AH_EINVAL
    finally:
        for b in (fresh, into, wrong):
            ah.ah_batch_free(b)


def test_fasta_pack_refuses_text_without_records(ah_ctx):
    ah, ctx = ah_ctx
    with pytest.raises(ah.AhError) as e:
        ah.ah_fasta_pack(ctx, b"ACGT\nACGT\n")
    assert e.value.status == ah.AH_EINVAL
    batch, names = ah.ah_fasta_pack(ctx, b">only a header")   # one empty record
    try:
        assert names == ["only a header"] and ah.ah_batch_view_get(batch)["n_bases"] == 0
    finally:
        ah.ah_batch_free(batch)


def test_fasta_pipeline_equals_direct_packing(ah_ctx):
    """The whole path on a batch packed from FASTA gives the oracle's sites and amplicons."""
    from paper_2511_00170_gb300.pipeline import Engine, Params
    from tests import compare

    wl = synth.random_small(31, n_records=6, len_lo=500, len_hi=20000, n_pairs=2, plant=3)
    lines = []
    for r in range(wl.n_records):
        s = wl.seq[wl.offsets[r]:wl.offsets[r + 1]].tobytes()
        lines.append(b">genome_%d some description" % r)
        lines += [s[i:i + 60] for i in range(0, len(s), 60)]
    text = b"\n".join(lines) + b"\n"
    eng = Engine(0)
    try:
        from paper_2511_00170_gb300 import ah

        batch, names = ah.ah_fasta_pack(eng.ctx, text)
        assert names == ["genome_%d some description" % r for r in range(wl.n_records)]
        out = eng.step(batch, Params.from_workload(wl))
        ah.ah_batch_free(batch)
    finally:
        eng.close()
    ref = oracle.run(wl)
    compare.assert_same_hits(out, ref)
    compare.assert_same_amplicons(out, ref, filtered=wl.tm.min_tm is not None)
    compare.assert_same_sequences(out, ref)


def _random_fastq(seed: int, n_records: int, crlf: bool) -> bytes:
    st = synth.Stream(synth.make_key(seed, 4322, 0))
    nl = b"\r\n" if crlf else b"\n"
    out = bytearray()
    for r in range(n_records):
        name = "read%d " % r + "".join(st.choice("abc XYZ:0123/") for _ in range(st.choice([3, 40, 6000])))
        L = st.choice([0, 1, 100, 150, 5000, 40000])
        seq = "".join(st.choice("ACGTACGTNacgt") for _ in range(L))
        qual = "".join(chr(st.randint(33, 74)) for _ in range(L))   # may start with '@' or '+'
        out += b"@" + name.encode() + nl + seq.encode() + nl + (b"+" if st.randint(0, 1) else b"+" + name.encode()) + nl
        out += qual.encode() + nl
    if st.randint(0, 1):
        out += nl + nl   # empty lines after the last record
    elif out.endswith(nl):
        out = out[: -len(nl)]
    return bytes(out)


@pytest.mark.parametrize("seed,n_records,crlf,on_device", [(1, 1, False, False), (2, 30, True, False),
                                                           (3, 50, False, True), (4, 9, True, True)])
def test_fastq_pack_matches_oracle(ah_ctx, seed, n_records, crlf, on_device):
    import torch

    ah, ctx = ah_ctx
    text = _random_fastq(seed, n_records, crlf)
    names, seqs, quals = oracle.parse_fastq(text)
    assert len(names) == n_records
    if on_device:
        d = torch.frombuffer(bytearray(text), dtype=torch.uint8).cuda()
        batch, q, got_names = ah.ah_fastq_pack(ctx, d.data_ptr(), n_bytes=len(text))
    else:
        batch, q, got_names = ah.ah_fastq_pack(ctx, text)
    lens = np.array([len(s) for s in seqs], dtype=np.uint64)
    ref = ah.ah_pack_batch(ctx, np.frombuffer(b"".join(seqs) or b"\0", dtype=np.uint8),
                           np.concatenate([[0], np.cumsum(lens)]).astype(np.int64))
    try:
        assert got_names == names
        assert _batch_bytes(ah, batch) == _batch_bytes(ah, ref)
        got_q, off = ah.ah_quals_copy(q)
        assert got_q == b"".join(quals)
        assert list(off) == list(np.concatenate([[0], np.cumsum([len(x) for x in quals])]))
    finally:
        ah.ah_batch_free(batch)
        ah.ah_batch_free(ref)
        ah.ah_quals_free(q)


@pytest.mark.parametrize("text", [b"ACGT\nACGT\n+\nIIII\n", b"@r\nACGT\n+\nIII\n",
                                  b"@r\nACGT\n+\nIIII\nnot a header\nAC\n+\nII\n",
                                  b"@r\n" + b"A" * 100000 + b"\n+\n\n"])   # bases over half the text
def test_fastq_pack_refuses_malformed(ah_ctx, text):
    ah, ctx = ah_ctx
    with pytest.raises(ah.AhError) as e:
        ah.ah_fastq_pack(ctx, text)
    assert e.value.status == ah.AH_EINVAL


@pytest.mark.parametrize("trim", [False, True])
def test_fastq_qualities_follow_the_amplicons(ah_ctx, trim):
    """The whole path on FASTQ input: the sites and amplicons of the oracle, and every kept amplicon's
    qualities those of its sequence field (reversed for RF); then the FASTQ writer's records."""
    from paper_2511_00170_gb300.pipeline import Engine, Params
    from tests import compare

    wl = synth.random_small(41 + trim, n_records=5, len_lo=500, len_hi=20000, n_pairs=2, plant=3, trim=trim)
    wl.orient_mask = 15
    st = synth.Stream(synth.make_key(7, 4323, 0))
    quals = []
    lines = []
    for r in range(wl.n_records):
        s = wl.seq[wl.offsets[r]:wl.offsets[r + 1]].tobytes()
        qv = bytes(st.randint(33, 74) for _ in range(len(s)))
        quals.append(qv)
        lines += [b"@genome_%d" % r, s, b"+", qv]
    text = b"\n".join(lines) + b"\n"
    eng = Engine(0)
    try:
        from paper_2511_00170_gb300 import ah

        batch, q, names = ah.ah_fastq_pack(eng.ctx, text)
        p = Params.from_workload(wl)
        hits, amps = eng.step(batch, p, copy_out=False)
        try:
            ah.ah_extract_qualities(eng.ctx, q, batch, eng.primers(p), hits, amps)
            ah.ah_ctx_synchronize(eng.ctx)
            from paper_2511_00170_gb300.pipeline import Output

            h = ah.ah_hits_copy(hits)
            a = ah.ah_amplicons_copy(amps)
            arena, off = ah.ah_amplicons_seq_copy(amps)
            qarena = ah.ah_amplicons_qual_copy(amps, len(arena))
            out = Output(h, a, arena, off)
        finally:
            ah.ah_hits_free(hits)
            ah.ah_amplicons_free(amps)
            ah.ah_quals_free(q)
            ah.ah_batch_free(batch)
    finally:
        eng.close()
    ref = oracle.run(wl)
    compare.assert_same_hits(out, ref)
    compare.assert_same_sequences(out, ref)
    kept = ref.amps[ref.keep]
    ref_q = dict(zip(compare.oracle_amp_keys(ref.hits, kept), oracle.amplicon_qualities(wl, ref.hits, kept, quals)))
    keys = compare.gpu_amp_keys(out)
    assert len(keys) == len(kept) > 0
    for m, k in enumerate(keys):
        assert qarena[int(off[5 * m]):int(off[5 * m + 1])] == ref_q[k], k
    fq = ah.ah_amplicons_fastq(a, arena, qarena, off, names)
    assert fq.count(b"\n+\n") == len(a)


def test_fasta_pack_host_text_in_several_chunks(ah_ctx):
    """Host text longer than one 256 MiB copy chunk is parsed chunk by chunk as it lands; records,
    a header line and a sequence line that cross chunk boundaries come out as from the oracle."""
    ah, ctx = ah_ctx
    rng = np.random.default_rng(11)
    chunk = 256 << 20
    parts, pos, r = [], 0, 0

    def record(name: bytes, L: int, width: int):
        nonlocal pos, r
        seq = rng.choice(np.frombuffer(b"ACGTACGTN", dtype=np.uint8), L)
        rows = [seq[i:i + width].tobytes() for i in range(0, L, width)] if width else [seq.tobytes()]
        txt = b">" + name + b"\n" + b"\n".join(rows) + b"\n"
        parts.append(txt)
        pos += len(txt)
        r += 1

    while pos < chunk - 30000:                       # ordinary records up to just before the first boundary
        record(b"rec%d" % r, int(rng.integers(1000, 3_000_000)), 80)
    parts.append(b"\n" * (chunk - 10000 - pos))      # empty lines: the next header starts 10,000 bytes before it
    pos = chunk - 10000
    record(b"long header " + b"x" * 20000, 5000, 60)  # its header crosses the boundary
    while pos < 2 * chunk - 50:
        record(b"rec%d" % r, int(rng.integers(1000, 3_000_000)), 0)   # one-line records cross the second
    record(b"last", 777, 70)
    text = b"".join(parts)
    assert len(text) > 2 * chunk
    names, seqs = oracle.parse_fasta(text)
    batch, got_names = ah.ah_fasta_pack(ctx, text)
    lens = np.array([len(s) for s in seqs], dtype=np.uint64)
    ref = ah.ah_pack_batch(ctx, np.frombuffer(b"".join(seqs), dtype=np.uint8),
                           np.concatenate([[0], np.cumsum(lens)]).astype(np.int64))
    try:
        assert got_names == names
        assert _batch_bytes(ah, batch) == _batch_bytes(ah, ref)
    finally:
        ah.ah_batch_free(batch)
        ah.ah_batch_free(ref)


def test_fastq_pack_host_text_in_several_chunks(ah_ctx):
    """FASTQ host text longer than two 256 MiB copy chunks is parsed chunk by chunk as it lands; a
    header line that crosses the first boundary and a sequence line that crosses the second come
    out as from the oracle, with every record's qualities."""
    ah, ctx = ah_ctx
    rng = np.random.default_rng(12)
    chunk = 256 << 20
    parts, pos = [], 0
    letters = np.frombuffer(b"ACGTACGTNacgt", dtype=np.uint8)

    def record(name: bytes, L: int):  # 2 L + len(name) + 6 bytes
        nonlocal pos
        txt = (b"@" + name + b"\n" + rng.choice(letters, L).tobytes() + b"\n+\n" +
               rng.integers(33, 75, L, dtype=np.uint8).tobytes() + b"\n")
        parts.append(txt)
        pos += len(txt)

    while pos < chunk - 5_000_000:
        record(b"read%d" % len(parts), int(rng.integers(100, 2_000_000)))
    rem = chunk - 10000 - pos                       # a filler record ends 10,000 bytes before the boundary
    name = b"f" if (rem - 7) % 2 == 0 else b"fg"
    record(name, (rem - 6 - len(name)) // 2)
    assert pos == chunk - 10000
    record(b"long header " + b"x" * 20000, 5000)    # its header line crosses the first boundary
    while pos < 2 * chunk - 5_000_000:
        record(b"read%d" % len(parts), int(rng.integers(100, 2_000_000)))
    record(b"s", 2 * chunk - pos - 3 + 1000)          # its sequence line crosses the second by 1,000 bytes
    record(b"last", 777)
    text = b"".join(parts)
    assert len(text) > 2 * chunk
    names, seqs, quals = oracle.parse_fastq(text)
    batch, q, got_names = ah.ah_fastq_pack(ctx, text)
    lens = np.array([len(s) for s in seqs], dtype=np.uint64)
    ref = ah.ah_pack_batch(ctx, np.frombuffer(b"".join(seqs), dtype=np.uint8),
                           np.concatenate([[0], np.cumsum(lens)]).astype(np.int64))
    try:
        assert got_names == names
        assert _batch_bytes(ah, batch) == _batch_bytes(ah, ref)
        got_q, off = ah.ah_quals_copy(q)
        assert got_q == b"".join(quals)
        assert list(off) == list(np.concatenate([[0], np.cumsum([len(x) for x in quals])]))
    finally:
        ah.ah_batch_free(batch)
        ah.ah_batch_free(ref)
        ah.ah_quals_free(q)


def test_fasta_and_fastq_files(ah_ctx, tmp_path):
    """The file front end gives the batch, names and qualities of the same text passed in memory;
    a missing file is refused with its name in the message."""
    ah, ctx = ah_ctx
    text = _random_fasta(11, 30, False, True)
    path = tmp_path / "genomes.fa"
    path.write_bytes(text)
    b_mem, n_mem = ah.ah_fasta_pack(ctx, text)
    b_file, n_file = ah.ah_fasta_pack_file(ctx, str(path))
    try:
        assert n_mem == n_file and len(n_file) > 0
        assert _batch_bytes(ah, b_mem) == _batch_bytes(ah, b_file)
    finally:
        ah.ah_batch_free(b_mem)
        ah.ah_batch_free(b_file)
    st = synth.Stream(synth.make_key(12, 4321, 0))
    recs = []
    for r in range(50):
        seq = "".join(st.choice("ACGTN") for _ in range(st.randint(0, 400)))
        qual = "".join(chr(33 + st.randint(0, 40)) for _ in seq)
        recs.append(f"@read{r} x\n{seq}\n+\n{qual}\n")
    fq = "".join(recs).encode()
    fq_path = tmp_path / "reads.fq"
    fq_path.write_bytes(fq)
    b1, q1, names1 = ah.ah_fastq_pack(ctx, fq)
    b2, q2, names2 = ah.ah_fastq_pack_file(ctx, str(fq_path))
    try:
        assert names1 == names2
        assert _batch_bytes(ah, b1) == _batch_bytes(ah, b2)
        qa, oa = ah.ah_quals_copy(q1)
        qb, ob = ah.ah_quals_copy(q2)
        assert qa == qb and np.array_equal(oa, ob)
    finally:
        for b in (b1, b2):
            ah.ah_batch_free(b)
        for q in (q1, q2):
            ah.ah_quals_free(q)
    with pytest.raises(ah.AhError) as e:
        ah.ah_fasta_pack_file(ctx, str(tmp_path / "missing.fa"))
    assert e.value.status == ah.AH_EINVAL and "missing.fa" in str(e.value)
