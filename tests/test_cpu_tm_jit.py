"""The generated degenerate-site Tm kernel compiles for every chain shape (NVRTC on the host, no
device): degenerate runs at either end and inside, positions two apart and further, three-choice
codes, concrete primers, primers of 2, 3 and 32 nt, repeated primers, sets of several pairs."""
import pytest

from paper_2511_00170_gb300 import ah

SETS = [
    ["SRNNAWCRWYAAGTSACC", "ATCWKSRANTMRRNATAA"],
    ["NNRYTGACCGTAGSAN", "NAGYCGATWKSGNACT"],
    ["BDTGACCGHVAGTCAN", "VHGYCGATWASGTACB", "RAYASAKAMAWAGTCC", "TGYARAYCAGATCACG"],
    ["ACGTTGCAGGTACCAT", "TTGGCCAAGCTAGCTA", "GACNTGAGCTAC", "TCAGGRTTCMAG"],
    ["ACGTRYKMACGTSWBDACGTHVGGACGTACGT", "TGCAACGTAGCTAGCTNNAGCTAGGCATGCAA"],
    ["AC", "NG", "ACG", "NNN", "RAN", "GCA"],
    ["GCTRACTAGCCATGWTCAG", "TTGACRSTAGCATGTCAGCA", "GCTRACTAGCCATGWTCAG", "TTGACRSTAGCATGTCAGCA"],
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.mark.parametrize("primers", SETS, ids=[str(i) for i in range(len(SETS))])
def test_generated_tm_kernel_compiles(primers):
    st, log = ah.ah_tm_kernel_check(primers, 103)
    assert st == 0, log


def test_bad_arguments():
    assert ah.ah_tm_kernel_check(["ACGTX"], 103)[0] == ah.AH_EINVAL
    assert ah.ah_tm_kernel_check(["A"], 103)[0] == ah.AH_EINVAL
    assert ah.ah_tm_kernel_check(["A" * 33], 103)[0] == ah.AH_EINVAL
