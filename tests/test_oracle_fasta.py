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
