"""The bit-sliced scan logic generated for a primer set (IUPAC plane selection, funnel shifts, the
carry-save counter tree and clamp terms as LOP3 truth tables), run on the CPU, equals an exact
per-position mismatch count and clamp check on random data, and every window its first phase
(clamp and most selective positions, after which a warp may skip the rest) fails does fail.  The
generic kernel's pattern table (per-position mismatch functions in algebraic normal form, the
evaluation order, the counter width), run through the generic kernel's equations with its warp
early exit, gives the same words.  No GPU is needed: everything is executed with numpy."""
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
    if not os.path.exists(exe) or os.path.getmtime(exe) < max(os.path.getmtime(os.path.join(lib, "libah.so")),
                                                              os.path.getmtime(src)):
        cuda_inc = "/usr/local/cuda/include"
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", cuda_inc, src, "-o", exe, "-L", lib, "-lah",
                               f"-Wl,-rpath,{lib}"])
    def run(k, c, prims, gen=False, shift=0, windows=1024, queue=0, persistent=0, min_blocks=0, compile=False,
            ops=False):
        args = (["gen"] if gen else []) + (["compile"] if compile else []) + (["ops"] if ops else [])
        args += [f"shift={shift}", f"windows={windows}", f"queue={queue}", f"persistent={persistent}",
                 f"min_blocks={min_blocks}", str(k), str(c)]
        return subprocess.run([exe] + args + prims, text=True, capture_output=True, check=not compile).stdout

    return run


CASES = [(2, 3, ["AGATACCKWCAACAACTGC", "CTCCTCGTATAWTMTCRACC"]), (0, 0, ["ACGTACGT"]),
         (1, 2, ["ACGRYSWKMBDHVN"]), (3, 3, ["NNNNACGTNNNNACGTAC"]), (5, 1, ["ACGTAGCTAGCTAGCATCGATCGATCGATCGA"]),
         (7, 0, ["AGCTTGACCGTAGGCATTAC"]), (15, 3, ["AGCTTGACCGTAGGCATTAC"]), (2, 20, ["AGCTTGACCGTAGGCATTAC"]),
         (4, 4, ["ACGTNACGTNACGTNACGTN"]), (6, 3, ["RRRRRRRRRRYYYYYYYYYY"]), (0, 2, ["AC"]), (1, 0, ["NN"])]


def _check(dump, k, clamp, primers, seed, n=2000, shift=0, windows=1024, queue=0):
    src = dump(k, clamp, primers, shift=shift, windows=windows, queue=queue)
    rng = np.random.default_rng(seed)
    planes = [rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32) for _ in range(4)]
    _check_planes(src, k, clamp, primers, planes)
    _check_planes(src, k, clamp, primers, _planted_planes(primers, k, clamp, n // 2, seed))


def _check_planes(src, k, clamp, primers, planes):
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


@pytest.mark.parametrize("shift", [1, 2])
@pytest.mark.parametrize("k,clamp,primers", CASES[:6])
def test_generated_logic_multiply_shifts(dump, k, clamp, primers, shift):
    """Shift modes 1 and 2 align the planes with multiply-adds (all of them, or every other one)
    instead of funnel shifts; the words are the same."""
    src = dump(k, clamp, primers, shift=shift)
    assert "mad.hi.u32" in src or "fshr(" not in src
    _check(dump, k, clamp, primers, 2, shift=shift)


@pytest.mark.parametrize("windows", [1, 64, 4096, 1 << 20])
@pytest.mark.parametrize("k,clamp,primers", CASES[:5] + CASES[8:10])
def test_generated_logic_phase_splits(dump, k, clamp, primers, windows):
    """The phase split is drawn by least expected work for a number of windows per warp vote: from
    1 (phase one as short as it gets) to 2^20 (one phase for most patterns), the words are exact and
    phase one never fails a matching window."""
    _check(dump, k, clamp, primers, 3, windows=windows)


def test_phase_split_follows_the_vote_width(dump):
    """For the bench pair (k=3, clamp 3) the split moves positions from phase two to phase one as the
    vote covers more windows (phase two then runs in more warps): the gates after the first vote
    never grow, and shrink from 1 window per vote to 2^20."""
    primers = ["AGATACCKWCAACAACTGC", "CTCCTCGTATAWTMTCRACC"]

    def phase_two_gates(windows):
        src = dump(3, 3, primers, windows=windows)
        body = src[src.index("const u32 lo0 = a.x"):src.index("if (__builtin_expect")]
        first_vote = body.find("__any_sync(__activemask()")
        return 0 if first_vote < 0 else body[first_vote:].count("lop3.b32")

    gates = [phase_two_gates(w) for w in (1, 64, 1024, 4096, 1 << 20)]
    assert all(x >= y for x, y in zip(gates, gates[1:])), gates
    assert gates[0] > gates[-1], gates


@pytest.mark.parametrize("k,clamp,primers", CASES[:4])
def test_generated_logic_candidate_queue(dump, k, clamp, primers):
    """With candidates queued per warp the circuit is the same and hands its words to the queue."""
    src = dump(k, clamp, primers, queue=1)
    assert "push4(" in src and "drain(P, first" in src
    _check(dump, k, clamp, primers, 4, queue=1)


@pytest.mark.parametrize("queue", [0, 1])
@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("shift,min_blocks", [(0, 0), (1, 4), (2, 0)])
def test_scan_kernel_variants_compile(dump, queue, persistent, shift, min_blocks):
    """Every form the autotuner may build compiles for sm_103a (NVRTC on the host, no device): one
    pair and the 8-pair batched set (inlined and called emission), each shift mode, the register
    bound, persistent CTAs, the candidate queue."""
    one = ["AGATACCKWCAACAACTGC", "CTCCTCGTATAWTMTCRACC"]
    eight = ["CGATANRNCGCGCCRCATMGTA", "MYGTGCTGYCACAACRCGA", "GTYAGCAAWGCACTCGMAAC", "GGCGMCGCGGGTYACRGTTGA",
             "CNGRRTATATSARCWGTATC", "CTAACCGGTAAACACTCACGA", "AGCGCTCAGTACAGCTAT", "TGCARTGAATCCTCWGCAGCCT",
             "GTRTGGGAGTGGTRAGTCGNTTACA", "CAGCAGTTCGGRTGCTCTGG", "CCGGCGTGTAGATCCTGTGATTA",
             "GGGCGTKTAGTGTSTGTTGTACACT", "AGGGSMGMAAGARARCMCGA", "TTAGCACWGATTTSGAACCAG", "CACKANCRKACCRCCCACA",
             "SGKGAATAGTTTARWTGTAG"]
    for prims in (one, eight):
        out = dump(2, 3, prims, shift=shift, queue=queue, persistent=persistent, min_blocks=min_blocks, compile=True)
        assert out.startswith("compiled "), out[:2000]


def test_bench_tables_describe_the_generated_circuits(dump):
    """bench.py keys its measured ALU-pipe and DRAM figures by circuit size.  The generator still
    builds the circuits they were measured on: the bench pair at 1,024 windows per vote, 186
    LOP3/SHF per 32 positions; the 8-pair batched set (k = i mod 4) at 4,096 windows (the
    autotuner's choice), 996, and at 1,024, 1,030."""
    import bench

    plain = ["AGATACCKWCAACAACTGC", "CTCCTCGTATAWTMTCRACC"]
    assert int(dump(3, 3, plain, ops=True)) == 186
    wl = synth.batched(n_genomes=3)
    batched = [f"{p}:{k}" for f, r, k in zip(wl.fwd, wl.rev, wl.k) for p in (f, r)]
    assert int(dump(0, wl.clamp, batched, windows=4096, ops=True)) == 996
    assert int(dump(0, wl.clamp, batched, windows=1024, ops=True)) == 1030
    assert 186 in bench.SCAN_PIPE and (186, 256, 8, 0, 0) in bench.SCAN_TRAFFIC
    assert (996, 4) in bench.SCAN_PIPE and (996, 128, 8, 0, 0) in bench.SCAN_TRAFFIC


@pytest.mark.parametrize("seed", range(8))
def test_generated_logic_random_primer_sets(dump, seed):
    st = synth.Stream(synth.make_key(seed, 4242, 0))
    L = st.randint(2, 32)
    clamp = st.randint(0, min(L, 6))
    k = st.randint(0, min(L, 15))
    prims = [synth.random_primer(st, st.randint(max(2, clamp), 32) if i else L, st.randint(0, 8), clamp,
                                 "RYSWKMBDHVN") for i in range(st.randint(1, 3))]
    _check(dump, k, clamp, prims, seed, n=600)


def _generic_failure_words(table, lo0, hi0, lo1, hi1):
    """The generic kernel's pass test per pattern, lanes of 32 words as warps (early exit after the
    clamp and every fourth counted position when no window of the warp is left)."""
    lines = table.strip().splitlines()
    out, i = [], 0
    ones = np.uint32(0xFFFFFFFF)
    while i < len(lines):
        L, k, n_eval, n_clamp, width, *_ = (int(v) for v in lines[i].split())
        pos = [tuple(int(v) for v in ln.split()) for ln in lines[i + 1:i + 1 + n_eval]]
        i += 1 + n_eval
        res = np.zeros(len(lo0), dtype=np.uint32)
        for w0 in range(0, len(lo0), 32):
            sl = slice(w0, w0 + 32)
            a_lo, a_hi = lo0[sl].astype(np.uint64), hi0[sl].astype(np.uint64)
            b_lo, b_hi = lo1[sl].astype(np.uint64), hi1[sl].astype(np.uint64)
            lo64, hi64 = a_lo | (b_lo << np.uint64(32)), a_hi | (b_hi << np.uint64(32))

            def mismatch(p):
                j, c0, c1, c2, c3 = p
                lo = ((lo64 >> np.uint64(j)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
                hi = ((hi64 >> np.uint64(j)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
                c0, c1, c2, c3 = (np.uint32(c) for c in (c0, c1, c2, c3))
                return ((lo & ((hi & c3) ^ c1)) ^ (hi & c2)) ^ c0

            fail = np.zeros(len(lo64), dtype=np.uint32)
            for p in pos[:n_clamp]:
                fail |= mismatch(p)
            if not np.any(~fail):
                continue
            c = [np.zeros(len(lo64), dtype=np.uint32) for _ in range(max(width, 1))]
            stopped = False
            for n, p in enumerate(pos[n_clamp:], start=1):
                x = mismatch(p)
                if width == 0:
                    fail |= x
                else:
                    carry = x
                    for w in range(width):
                        nc = c[w] & carry
                        c[w] ^= carry
                        carry = nc
                    fail |= carry
                if n % 4 == 0 and not np.any(~fail):
                    stopped = True
                    break
            if stopped:
                continue
            T = k + 1
            if width > 0 and T < (1 << width):
                ge = np.full(len(lo64), ones, dtype=np.uint32)
                for w in range(width):
                    ge = (c[w] & ge) if (T >> w) & 1 else (c[w] | ge)
                fail |= ge
            res[sl] = ~fail
        out.append(~res)  # failure words
    return out


def _planted_planes(primers, k, clamp, n, seed):
    """Planes (lo, hi of group g; lo, hi of group g + 1) of a random sequence holding many planted
    instances of the patterns with about k mismatches (k - 1 to k + 2, now and then one in the
    clamp), so that the count comparison decides many windows."""
    rng = np.random.default_rng(seed)
    seq = rng.integers(0, 4, 32 * (n + 1))
    pats = []
    for p in primers:
        rc = "".join(scan_emulator.COMP[c] for c in reversed(p))
        pats += [(p, set(range(len(p) - clamp, len(p)))), (rc, set(range(clamp)))]
    for _ in range(n // 2):
        pat, cl = pats[rng.integers(len(pats))]
        at = int(rng.integers(0, len(seq) - len(pat)))
        bases = [scan_emulator.SETS[ch][rng.integers(len(scan_emulator.SETS[ch]))] for ch in pat]
        free = [j for j, ch in enumerate(pat) if ch != "N" and j not in cl]
        m = min(len(free), max(0, k - 1 + int(rng.integers(0, 4))))
        mis = list(rng.choice(free, m, replace=False)) if m else []
        if cl and rng.random() < 0.1:
            mis.append(int(rng.choice(sorted(cl))))
        for j in mis:
            others = [b for b in "ACGT" if b not in scan_emulator.SETS[pat[j]]]
            if others:
                bases[j] = others[rng.integers(len(others))]
        seq[at:at + len(pat)] = [scan_emulator.CODE[b] for b in bases]
    bits = lambda b: np.packbits(((seq >> b) & 1).astype(np.uint8).reshape(-1, 32)[:, ::-1], axis=1) \
        .view(">u4").ravel().astype(np.uint32)
    lo, hi = bits(0), bits(1)
    return [lo[:-1].copy(), hi[:-1].copy(), lo[1:].copy(), hi[1:].copy()]


def _check_generic(dump, k, clamp, primers, seed, n=1024):
    table = dump(k, clamp, primers, gen=True)
    planes = _planted_planes(primers, k, clamp, n, seed)
    got = _generic_failure_words(table, *planes)
    want = scan_emulator.exact_failure_words(primers, k, clamp, *planes)
    assert len(got) == len(want) == 2 * len(primers)
    for q, (g, w) in enumerate(zip(got, want)):
        assert np.array_equal(g, w), f"pattern {q}: {int(np.count_nonzero(g != w))} words differ"


@pytest.mark.parametrize("k,clamp,primers", CASES)
def test_generic_table_fixed_cases(dump, k, clamp, primers):
    _check_generic(dump, k, clamp, primers, 3)


@pytest.mark.parametrize("seed", range(6))
def test_generic_table_random_primer_sets(dump, seed):
    st = synth.Stream(synth.make_key(seed, 4243, 0))
    L = st.randint(2, 32)
    clamp = st.randint(0, min(L, 6))
    k = st.randint(0, min(L, 15))
    prims = [synth.random_primer(st, st.randint(max(2, clamp), 32) if i else L, st.randint(0, 8), clamp,
                                 "RYSWKMBDHVN") for i in range(st.randint(1, 3))]
    _check_generic(dump, k, clamp, prims, seed, n=512)
