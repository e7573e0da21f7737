"""The oracle's FASTA parser on a hand-written text: names, sequences, line breaks and blanks
dropped, lines before the first header ignored, empty records kept (the input format of the
Abstract: FASTA packed into 2-bit batches)."""
import oracle


def test_parse_fasta_hand_example():
    text = (b"junk before any record\n"
            b">chr1 Escherichia coli\r\n"
            b"ACGTN\r\n"
            b"acg t\tRY\r\n"
            b"\r\n"
            b">empty\n"
            b">last one\n"
            b"GGG")
    names, seqs = oracle.parse_fasta(text)
    assert names == ["chr1 Escherichia coli", "empty", "last one"]
    assert seqs == [b"ACGTNacgtRY", b"", b"GGG"]


def test_parse_fasta_no_records():
    assert oracle.parse_fasta(b"ACGT\nACGT\n") == ([], [])


def test_parse_fastq_hand_example():
    text = (b"@read1 first\r\n"
            b"ACGTN\r\n"
            b"+\r\n"
            b"IIII#\r\n"
            b"@read2\n"
            b"\n"
            b"+read2\n"
            b"\n"
            b"@read3\n"
            b"GG\n"
            b"+\n"
            b"@I\n"
            b"\n\n")
    names, seqs, quals = oracle.parse_fastq(text)
    assert names == ["read1 first", "read2", "read3"]
    assert seqs == [b"ACGTN", b"", b"GG"]
    assert quals == [b"IIII#", b"", b"@I"]   # a quality line may start with '@'


def test_parse_fastq_refuses_malformed():
    """A record without its '@' header line, or with qualities of another length than its bases,
    is not FASTQ."""
    import pytest

    for text in (b"ACGT\nACGT\n+\nIIII\n", b"@r\nACGT\n+\nIII\n", b"@r\nAC\n+\nII\nnot a header\nAC\n+\nII\n"):
        with pytest.raises(AssertionError):
            oracle.parse_fastq(text)


def test_fastq_and_fasta_parsers_agree():
    """The same records written as FASTQ and as FASTA (one sequence line each) parse to the same
    names and sequences."""
    import random

    rnd = random.Random(7)
    fq, fa = bytearray(), bytearray()
    for r in range(40):
        name = b"read%d %s" % (r, bytes(rnd.choice(b"abc :/0") for _ in range(rnd.randint(0, 12))))
        seq = bytes(rnd.choice(b"ACGTNacgt") for _ in range(rnd.choice([0, 1, 7, 150])))
        qual = bytes(rnd.randint(33, 74) for _ in seq)
        fq += b"@" + name + b"\n" + seq + b"\n+\n" + qual + b"\n"
        fa += b">" + name + b"\n" + seq + b"\n"
    names_q, seqs_q, quals = oracle.parse_fastq(bytes(fq))
    names_a, seqs_a = oracle.parse_fasta(bytes(fa))
    assert names_q == names_a and seqs_q == seqs_a
    assert [len(q) for q in quals] == [len(s) for s in seqs_q]
