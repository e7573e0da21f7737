"""The bit-sliced scan logic generated for a primer set (IUPAC plane selection, funnel shifts, the
carry-save counter tree and clamp terms as LOP3 truth tables), run on the CPU, equals an exact
per-position mismatch count and clamp check on random data, and every window its first phase
(clamp and most selective positions, after which a warp may skip the rest) fails does fail.  No
GPU is needed: the generated statements are executed with numpy."""
import os
import subprocess

import numpy as np
import pytest

import synth
from tests import scan_emulator

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dump():
    import __graft_entry__

    __graft_entry__.build()
    exe = os.path.join(ROOT, "paper_2511_00170_gb300", "_build", "jit_dump")
    src = os.path.join(ROOT, "tests", "jit_dump.cpp")
    lib = os.path.join(ROOT, "paper_2511_00170_gb300")
    if not os.path.exists(exe) or os.path.getmtime(exe) < os.path.getmtime(os.path.join(lib, "libah.so")):
        cuda_inc = "/usr/local/cuda/include"
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", cuda_inc, src, "-o", exe, "-L", lib, "-lah",
                               f"-Wl,-rpath,{lib}"])
    return lambda k, c, prims: subprocess.check_output([exe, str(k), str(c)] + prims, text=True)


CASES = [(2, 3, ["AGATACCKWCAACAACTGC", "CTCCTCGTATAWTMTCRACC"]), (0, 0, ["ACGTACGT"]),
         (1, 2, ["ACGRYSWKMBDHVN"]), (3, 3, ["NNNNACGTNNNNACGTAC"]), (5, 1, ["ACGTAGCTAGCTAGCATCGATCGATCGATCGA"]),
         (7, 0, ["AGCTTGACCGTAGGCATTAC"]), (15, 3, ["AGCTTGACCGTAGGCATTAC"]), (2, 20, ["AGCTTGACCGTAGGCATTAC"]),
         (4, 4, ["ACGTNACGTNACGTNACGTN"]), (6, 3, ["RRRRRRRRRRYYYYYYYYYY"]), (0, 2, ["AC"]), (1, 0, ["NN"])]


def _check(dump, k, clamp, primers, seed, n=2000):
    src = dump(k, clamp, primers)
    rng = np.random.default_rng(seed)
    planes = [rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32) for _ in range(4)]
    phase_a = []
    got = scan_emulator.failure_words(src, *planes, phase_a=phase_a)
    want = scan_emulator.exact_failure_words(primers, k, clamp, *planes)
    assert len(got) == len(want) == 2 * len(primers)
    for q, (g, w) in enumerate(zip(got, want)):
        assert np.array_equal(g, w), f"pattern {q}: {int(np.count_nonzero(g != w))} words differ"
    # the warp vote may skip phase B only where phase A already says "fail": every window phase A
    # fails must fail in the end
    for q, (a, w) in enumerate(zip(phase_a, want)):
        assert not np.any(a & ~w), f"pattern {q}: phase A fails a window that matches"


@pytest.mark.parametrize("k,clamp,primers", CASES)
def test_generated_logic_fixed_cases(dump, k, clamp, primers):
    _check(dump, k, clamp, primers, 1)


@pytest.mark.parametrize("seed", range(8))
def test_generated_logic_random_primer_sets(dump, seed):
    st = synth.Stream(synth.make_key(seed, 4242, 0))
    L = st.randint(2, 32)
    clamp = st.randint(0, min(L, 6))
    k = st.randint(0, min(L, 15))
    prims = [synth.random_primer(st, st.randint(max(2, clamp), 32) if i else L, st.randint(0, 8), clamp,
                                 "RYSWKMBDHVN") for i in range(st.randint(1, 3))]
    _check(dump, k, clamp, prims, seed, n=600)
