"""CPU execution of the straight-line logic of a generated scan kernel.

The generated kernel computes, for 32 positions at once, a failure word per pattern from the two
code-bit planes of two consecutive groups.  This module runs exactly those statements with numpy:
plane definitions, funnel shifts (or their multiply-add form), LOP3 instructions (evaluated from
their truth tables), and
compares each failure word with an exact per-position mismatch count and clamp check.
"""
import re

import numpy as np

M = np.uint32(0xFFFFFFFF)
SETS = {"A": "A", "C": "C", "G": "G", "T": "T", "R": "AG", "Y": "CT", "S": "CG", "W": "AT", "K": "GT", "M": "AC",
        "B": "CGT", "D": "AGT", "H": "ACT", "V": "ACG", "N": "ACGT"}
CODE = {"A": 0, "C": 1, "T": 2, "G": 3}
COMP = {"A": "T", "C": "G", "G": "C", "T": "A", "R": "Y", "Y": "R", "S": "S", "W": "W", "K": "M", "M": "K", "B": "V",
        "V": "B", "D": "H", "H": "D", "N": "N"}


def fshr(a, b, s):
    s = int(s)
    return a if s == 0 else ((a >> np.uint32(s)) | (b << np.uint32(32 - s))) & M


def _expr(e, env):
    e = e.replace("0xffffffffu", "M")
    e = re.sub(r"\b(\d+)u\b", r"\1", e)
    e = re.sub(r"~(\w+)", r"(M ^ \1)", e).replace("~(", "M ^ (")
    return np.asarray(eval(e, {"np": np, "M": M, "fshr": fshr}, env), dtype=np.uint32)


def failure_words(src, lo0, hi0, lo1, hi1, phase_a=None):
    """Run the generated body; returns the failure word of every pattern.  With phase_a (a list),
    also appends each pattern's phase-A word (the word before the warp-vote branch) to it."""
    body = src[src.index("const u32 lo0 = a.x"):src.index("if (__builtin_expect")]
    env = {"lo0": lo0, "hi0": hi0, "lo1": lo1, "hi1": hi1}
    zero = np.zeros_like(lo0)
    for line in body.split("\n"):
        m = re.match(r"\s*const u32 (\w+) = (.*?);$", line)
        if m:
            if m.group(1) not in env:
                env[m.group(1)] = _expr(m.group(2), env)
            continue
        # a pattern's failure word: phase A's value, then (inside the warp-vote branch, which every
        # emulated lane takes) the final value after phase B; lanes whose windows all failed phase A
        # are left with phase A's word, which is already all ones
        m = re.match(r"\s*(u32 )?(f\d+) = (.*?);$", line)
        if m:
            env[m.group(2)] = zero | _expr(m.group(3), env)   # constants become one word per lane
            if m.group(1):
                env["phase_a_" + m.group(2)] = env[m.group(2)]
            continue
        # a shift by two multiply-adds: t = lo(w1 * m), then hi(w0 * m) + t (m = 2^(32 - j))
        m = re.match(r'\s*\{ u32 t_; asm\("mul.lo.u32 %0, %1, (\d+);" : "=r"\(t_\) : "r"\((\w+)\)\); '
                     r'asm\("mad.hi.u32 %0, %1, (\d+), %2;" : "=r"\((\w+)\) : "r"\((\w+)\), "r"\(t_\)\); \}', line)
        if m:
            m1, w1, m2, name, w0 = m.group(1, 2, 3, 4, 5)
            t = (env[w1].astype(np.uint64) * np.uint64(int(m1))) & np.uint64(0xFFFFFFFF)
            h = (env[w0].astype(np.uint64) * np.uint64(int(m2))) >> np.uint64(32)
            env[name] = ((h + t) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
            continue
        m = re.match(r'\s*u32 (\w+); asm\("lop3.b32 %0, %1, %2, %3, (0x[0-9a-f]+);" : "=r"\(\w+\) : '
                     r'"r"\((\w+)\), "r"\((\w+)\), "r"\((\w+)\)\);', line)
        if m:
            lut = int(m.group(2), 16)
            a, b, c = (zero if x == "0u" else env[x] for x in m.group(3, 4, 5))
            r = np.zeros_like(a)
            for idx in range(8):
                if (lut >> idx) & 1:
                    r |= (a if idx & 4 else M ^ a) & (b if idx & 2 else M ^ b) & (c if idx & 1 else M ^ c)
            env[m.group(1)] = r
    # the candidate words handed to the emission routine or the warp's queue, four patterns per call
    # (~f<q>, or 0u where the block of four has no pattern)
    names = []
    for args in re.findall(r"(?:emit4|push4)\(([^;]*?), \d+, (?:\(u32\)\(gl - first\), )?g, a, b, P[,)]", src):
        names += [x[1:] for x in (a.strip() for a in args.split(",")) if x != "0u"]
    if phase_a is not None:
        for f in names:
            phase_a.append(env.get("phase_a_" + f, env.get(f)))
    return [env[f] for f in names]


def exact_failure_words(primers, k, clamp, lo0, hi0, lo1, hi1):
    lo64 = lo0.astype(np.uint64) | (lo1.astype(np.uint64) << np.uint64(32))
    hi64 = hi0.astype(np.uint64) | (hi1.astype(np.uint64) << np.uint64(32))
    out = []
    for p in primers:
        rc = "".join(COMP[c] for c in reversed(p))
        for pat, cl in ((p, range(len(p) - clamp, len(p))), (rc, range(0, clamp))):
            word = np.zeros(len(lo0), dtype=np.uint32)
            for i in range(32):
                mism = np.zeros(len(lo0), dtype=np.int64)
                bad = np.zeros(len(lo0), dtype=bool)
                for j, ch in enumerate(pat):
                    code = ((lo64 >> np.uint64(i + j)) & np.uint64(1)) | \
                           (((hi64 >> np.uint64(i + j)) & np.uint64(1)) << np.uint64(1))
                    ok = np.zeros(len(lo0), dtype=bool)
                    for base in SETS[ch]:
                        ok |= code == CODE[base]
                    mism += ~ok
                    if j in cl:
                        bad |= ~ok
                word |= ((bad | (mism > k)).astype(np.uint32) << np.uint32(i))
            out.append(word)
    return out
