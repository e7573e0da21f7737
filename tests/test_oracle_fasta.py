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
