"""Seeded synthetic workloads for the in-silico PCR hot path.

This module draws inputs only: genome records (ASCII, with runs of N and tandem repeats),
degenerate IUPAC primer pairs, planted amplicon templates, and the run parameters of each
workload.  It contains none of the matching, pairing, melting-temperature or extraction
arithmetic; the oracle and the CUDA path each implement those on their own and are both fed
from here.

All randomness is counter based (SplitMix64 output function applied to key + counter), keyed
by (seed, tag, genome), so a workload is a pure function of its seed and size parameters.

Workloads (the stand-ins for the paper's AllTheBacteria genomes and its V1V9 / Titan / V3V4
primer pairs, which are not available here):

* ``plain_small``  -- 16 genomes, U(1,3) Mbp, GC 50 %, 0.5 % N in runs of 1-50, one pair
  (19 nt fwd with 2 degenerate codes, 20 nt rev with 3), 3 planted 250-300 bp templates per
  genome with 0-3 substitutions per binding site, k=2, clamp 3, window 50-2000, Tm filter 45 C.
* ``plain_scale``  -- 2,000 genomes, lognormal length (median 3.5 Mbp, sigma 0.4), per-genome
  GC ~ U(0.30,0.70), 1-15 planted 16S-like templates per genome (one 1.4-1.6 kbp interior per
  genome) with 0-4 substitutions per binding site, same pair, k=3, trimming, 16 nt barcodes.
* ``batched``      -- many genomes, log-uniform 10 kbp - 12 Mbp, 8 pairs of 17-26 nt with 0-6
  degenerate codes, k_i = i mod 4, 0-3 planted templates per genome.
* ``dense``        -- genomes as plain_scale, 30 % carrying tandem repeats (period 2-12,
  1-20 kbp), primers with up to 9 degenerate codes including N, window 50-5000, all four
  orientations.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED = 251100170
_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "_synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the bulk generator (plain C, no GPU) next to this file."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _get_lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u8p = ctypes.c_void_p
            lib.synth_fill_bases.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64]
            lib.synth_fill_bases.restype = None
            lib.synth_fill_nruns.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint32]
            lib.synth_fill_nruns.restype = ctypes.c_uint64
            lib.synth_nrun_list.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint32, u8p,
                                            u8p, ctypes.c_uint64]
            lib.synth_nrun_list.restype = ctypes.c_uint64
            lib.synth_fill_tandem.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
            lib.synth_fill_tandem.restype = None
            lib.synth_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_draw.restype = ctypes.c_uint64
            _lib = lib
    return _lib


# ----------------------------------------------------------------------------- counter RNG
def mix64(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def draw(key: int, i: int) -> int:
    return mix64(key + (i + 1) * _GOLDEN)


def make_key(seed: int, *tags: int) -> int:
    k = mix64(seed)
    for t in tags:
        k = mix64(k ^ ((t + 0x632BE59BD9B4E019) * 0xD6E8FEB86659FD93 & _M64))
    return k


class Stream:
    """Sequential view of one counter-based stream (for small, scalar draws)."""

    def __init__(self, key: int):
        self.key = key
        self.c = 0

    def u64(self) -> int:
        v = draw(self.key, self.c)
        self.c += 1
        return v

    def unit(self) -> float:
        return (self.u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """uniform integer in [lo, hi] inclusive"""
        return lo + self.u64() % (hi - lo + 1)

    def normal(self) -> float:
        u1 = max(self.unit(), 1e-300)
        u2 = self.unit()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def choice(self, seq):
        return seq[self.u64() % len(seq)]

    def sample(self, n: int, k: int) -> List[int]:
        """k distinct values from range(n) (partial Fisher-Yates)"""
        pool = list(range(n))
        for i in range(k):
            j = i + self.u64() % (n - i)
            pool[i], pool[j] = pool[j], pool[i]
        return pool[:k]


# Tags separating the streams of one workload.
T_LEN, T_GC, T_BASES, T_NRUN, T_PRIMER, T_PLANT, T_TANDEM, T_SUBSET = range(1, 9)

# IUPAC sets used only to draw concrete primer variants for planted templates.
_SETS = {"A": "A", "C": "C", "G": "G", "T": "T", "R": "AG", "Y": "CT", "S": "CG", "W": "AT",
         "K": "GT", "M": "AC", "B": "CGT", "D": "AGT", "H": "ACT", "V": "ACG", "N": "ACGT"}
_COMP = {"A": "T", "C": "G", "G": "C", "T": "A", "N": "N"}
DEGENERATE_CODES = "RYMKSWN"


def _revcomp_plain(s: str) -> str:
    return "".join(_COMP[c] for c in reversed(s))


@dataclass
class TmParams:
    Na: float = 50.0      # mM
    K: float = 0.0        # mM
    Tris: float = 0.0     # mM
    Mg: float = 0.0       # mM
    dNTPs: float = 0.0    # mM
    dnac1: float = 25.0   # nM
    dnac2: float = 25.0   # nM
    saltcorr: int = 5
    min_tm: Optional[float] = None   # None: annotate only, no filtering
    variants: int = 0     # degenerate Tm over 0: every concrete variant, 1: those matching the site
    selfcomp: int = 0     # 1: the duplexes are self-complementary (symmetry term, C = dnac1)
    nn_table: int = 0     # nearest-neighbour set (Biopython's numbering; 0 the default DNA_NN3)


@dataclass
class Planted:
    genome: int
    pos: int
    strand: int        # 0: template on the top strand, 1: reverse-complemented
    pair: int
    length: int
    subs_f: int
    subs_r: int


@dataclass
class Workload:
    name: str
    seq: np.ndarray                 # uint8 ASCII, all records concatenated
    offsets: np.ndarray             # int64, n_records + 1
    genome_ids: np.ndarray          # uint32, n_records
    fwd: List[str]
    rev: List[str]
    k: List[int]
    clamp: int
    min_len: int
    max_len: int
    orient_mask: int                # bit0 FR, bit1 RF, bit2 FF, bit3 RR
    tm: TmParams
    trim: bool
    fb_len: int
    rb_len: int
    planted: List[Planted] = field(default_factory=list)
    seed: int = SEED
    extract: bool = True            # the path writes amplicon sequences, barcodes and snippets

    @property
    def n_records(self) -> int:
        return len(self.offsets) - 1

    @property
    def total_bp(self) -> int:
        return int(self.offsets[-1])

    def record(self, i: int) -> np.ndarray:
        return self.seq[self.offsets[i]:self.offsets[i + 1]]

    def record_str(self, i: int) -> str:
        return self.record(i).tobytes().decode("ascii")

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def subset(self, records: Sequence[int]) -> "Workload":
        """A workload over a subset of the records (copied), same primers and parameters."""
        recs = list(records)
        lens = [int(self.offsets[i + 1] - self.offsets[i]) for i in recs]
        offs = np.zeros(len(recs) + 1, dtype=np.int64)
        offs[1:] = np.cumsum(lens)
        seq = np.empty(int(offs[-1]), dtype=np.uint8)
        for j, i in enumerate(recs):
            seq[offs[j]:offs[j + 1]] = self.record(i)
        return Workload(self.name + "-subset", seq, offs, self.genome_ids[recs].copy(), list(self.fwd),
                        list(self.rev), list(self.k), self.clamp, self.min_len, self.max_len,
                        self.orient_mask, self.tm, self.trim, self.fb_len, self.rb_len, [], self.seed, self.extract)


# ----------------------------------------------------------------------------- primers
def random_primer(st: Stream, length: int, n_degenerate: int, clamp: int, codes: str = DEGENERATE_CODES) -> str:
    bases = [st.choice("ACGT") for _ in range(length)]
    n_degenerate = min(n_degenerate, max(0, length - clamp))
    for p in st.sample(length - clamp, n_degenerate):
        bases[p] = st.choice(codes)
    return "".join(bases)


def concrete_variant(st: Stream, primer: str) -> str:
    return "".join(st.choice(_SETS[c]) for c in primer)


def substitute(st: Stream, s: str, n_subs: int) -> str:
    b = list(s)
    for p in st.sample(len(b), min(n_subs, len(b))):
        b[p] = st.choice([x for x in "ACGT" if x != b[p]])
    return "".join(b)


# ----------------------------------------------------------------------------- genomes
def _fill_genomes(seq: np.ndarray, offsets: np.ndarray, seed: int, gcs: Sequence[float],
                  n_frac: float, n_run_max: int, threads: int = 0) -> None:
    lib = _get_lib()
    n = len(offsets) - 1
    base = seq.ctypes.data

    def work(lo, hi):
        for g in range(lo, hi):
            a, b = int(offsets[g]), int(offsets[g + 1])
            lib.synth_fill_bases(base + a, b - a, make_key(seed, T_BASES, g), float(gcs[g]), 0)
            if n_frac > 0:
                lib.synth_fill_nruns(base + a, b - a, make_key(seed, T_NRUN, g), n_frac, n_run_max)

    threads = threads or min(16, os.cpu_count() or 1)
    chunk = max(1, (n + threads * 4 - 1) // (threads * 4))
    ts = [threading.Thread(target=work, args=(i, min(n, i + chunk))) for i in range(0, n, chunk)]
    # ctypes releases the GIL during the C calls, so the threads run in parallel
    for t in ts:
        t.start()
    for t in ts:
        t.join()


def _plant(seq: np.ndarray, offsets: np.ndarray, g: int, st: Stream, n_sites: int, fwd: str, rev: str,
           pair: int, interior_len_fn, subs_max: int, planted: List[Planted], interior: Optional[str] = None) -> None:
    a, b = int(offsets[g]), int(offsets[g + 1])
    glen = b - a
    if n_sites <= 0:
        return
    seg = glen // n_sites
    for s in range(n_sites):
        fv = concrete_variant(st, fwd)
        rv = concrete_variant(st, rev)
        sf = st.randint(0, subs_max)
        sr = st.randint(0, subs_max)
        fv = substitute(st, fv, sf)
        rv = substitute(st, rv, sr)
        mid = interior if interior is not None else "".join(st.choice("ACGT") for _ in range(interior_len_fn(st)))
        tmpl = fv + mid + _revcomp_plain(rv)
        strand = st.randint(0, 1)
        if strand:
            tmpl = _revcomp_plain(tmpl)
        if len(tmpl) + 2 > seg:
            continue
        off = s * seg + st.randint(0, seg - len(tmpl) - 1)
        seq[a + off:a + off + len(tmpl)] = np.frombuffer(tmpl.encode("ascii"), dtype=np.uint8)
        planted.append(Planted(g, off, strand, pair, len(tmpl), sf, sr))


T_INTERIOR = 9


def c_bases(n: int, key: int, gc: float = 0.5) -> str:
    """n iid bases drawn by the C filler (fast path for long template interiors)."""
    buf = np.empty(n, dtype=np.uint8)
    if n:
        _get_lib().synth_fill_bases(buf.ctypes.data, n, key, gc, 0)
    return buf.tobytes().decode("ascii")


def batched_templates(seed: int, lengths: Sequence[int], fwd: List[str], rev: List[str], subs_max: int = 3):
    """Planted templates of the batched workload: per genome 0-3 templates of one random pair,
    interiors of 200-1500 bases.  Returns (list of (genome, offset, bytes), planted records)."""
    out, planted = [], []
    n_pairs = len(fwd)
    for g, glen in enumerate(lengths):
        st = Stream(make_key(seed + 2, T_PLANT, g))
        n_sites = st.randint(0, 3)
        p = st.randint(0, n_pairs - 1)
        if n_sites == 0:
            continue
        seg = glen // n_sites
        for s in range(n_sites):
            fv = substitute(st, concrete_variant(st, fwd[p]), sf := st.randint(0, subs_max))
            rv = substitute(st, concrete_variant(st, rev[p]), sr := st.randint(0, subs_max))
            mid = c_bases(st.randint(200, 1500), make_key(seed + 2, T_INTERIOR, g * 8 + s))
            tmpl = fv + mid + _revcomp_plain(rv)
            strand = st.randint(0, 1)
            if strand:
                tmpl = _revcomp_plain(tmpl)
            if len(tmpl) + 2 > seg:
                continue
            off = s * seg + st.randint(0, seg - len(tmpl) - 1)
            out.append((g, off, tmpl.encode("ascii")))
            planted.append(Planted(g, off, strand, p, len(tmpl), sf, sr))
    return out, planted


def batched_lengths_and_primers(seed: int, n_genomes: int, len_lo: float, len_hi: float, n_pairs: int):
    st_len = Stream(make_key(seed + 2, T_LEN, 0))
    la, lb = math.log(len_lo), math.log(len_hi)
    lengths = [int(math.exp(la + (lb - la) * st_len.unit())) for _ in range(n_genomes)]
    st_gc = Stream(make_key(seed + 2, T_GC, 0))
    gcs = [0.30 + 0.40 * st_gc.unit() for _ in range(n_genomes)]
    pst = Stream(make_key(seed + 2, T_PRIMER, 0))
    fwd, rev = [], []
    for _ in range(n_pairs):
        fwd.append(random_primer(pst, pst.randint(17, 26), pst.randint(0, 6), 3))
        rev.append(random_primer(pst, pst.randint(17, 26), pst.randint(0, 6), 3))
    return lengths, gcs, fwd, rev


def _alloc(lengths: Sequence[int], out: Optional[np.ndarray]):
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(np.asarray(lengths, dtype=np.int64))
    total = int(offsets[-1])
    if out is not None:
        if out.dtype != np.uint8 or out.size < total:
            raise ValueError("out buffer too small")
        seq = out[:total]
    else:
        seq = np.empty(total, dtype=np.uint8)
    return seq, offsets


def plain_small(seed: int = SEED, n_genomes: int = 16, len_lo: int = 1_000_000, len_hi: int = 3_000_000,
                out: Optional[np.ndarray] = None) -> Workload:
    """16 genomes U(1,3) Mbp, one degenerate pair, k=2, Tm filter 45 C."""
    st_len = Stream(make_key(seed, T_LEN, 0))
    lengths = [st_len.randint(len_lo, len_hi) for _ in range(n_genomes)]
    seq, offsets = _alloc(lengths, out)
    _fill_genomes(seq, offsets, seed, [0.5] * n_genomes, 0.005, 50)
    pst = Stream(make_key(seed, T_PRIMER, 0))
    fwd = random_primer(pst, 19, 2, 3)
    rev = random_primer(pst, 20, 3, 3)
    planted: List[Planted] = []
    for g in range(n_genomes):
        st = Stream(make_key(seed, T_PLANT, g))
        _plant(seq, offsets, g, st, 3, fwd, rev, 0,
               lambda s: s.randint(250, 300) - len(fwd) - len(rev), 3, planted)
    return Workload("plain_small", seq, offsets, np.arange(n_genomes, dtype=np.uint32), [fwd], [rev], [2], 3,
                    50, 2000, 0b0011 | 0b1100, TmParams(min_tm=45.0), False, 0, 0, planted, seed)


def plain_scale(seed: int = SEED, n_genomes: int = 2000, median: float = 3.5e6, sigma: float = 0.4,
                out: Optional[np.ndarray] = None) -> Workload:
    """2,000 lognormal genomes (~7.6 Gbp), per-genome GC, 1-15 planted 16S-like sites, k=3, trim, barcodes."""
    st_len = Stream(make_key(seed + 1, T_LEN, 0))
    lengths = [max(1000, int(round(median * math.exp(sigma * st_len.normal())))) for _ in range(n_genomes)]
    st_gc = Stream(make_key(seed + 1, T_GC, 0))
    gcs = [0.30 + 0.40 * st_gc.unit() for _ in range(n_genomes)]
    seq, offsets = _alloc(lengths, out)
    _fill_genomes(seq, offsets, seed + 1, gcs, 0.005, 50)
    pst = Stream(make_key(seed, T_PRIMER, 0))        # the same pair as plain_small
    fwd = random_primer(pst, 19, 2, 3)
    rev = random_primer(pst, 20, 3, 3)
    planted: List[Planted] = []
    for g in range(n_genomes):
        st = Stream(make_key(seed + 1, T_PLANT, g))
        n_sites = st.randint(1, 15)
        ilen = st.randint(1400, 1600)
        interior = "".join(st.choice("ACGT") for _ in range(ilen))
        _plant(seq, offsets, g, st, n_sites, fwd, rev, 0, None, 4, planted, interior=interior)
    return Workload("plain_scale", seq, offsets, np.arange(n_genomes, dtype=np.uint32), [fwd], [rev], [3], 3,
                    50, 2000, 0b1111, TmParams(min_tm=None), True, 16, 16, planted, seed)


def batched(seed: int = SEED, n_genomes: int = 50_000, len_lo: float = 1e4, len_hi: float = 1.2e7,
            n_pairs: int = 8, out: Optional[np.ndarray] = None) -> Workload:
    """Many log-uniform genomes, 8 pairs of 17-26 nt with 0-6 degenerate codes, k_i = i mod 4."""
    lengths, gcs, fwd, rev = batched_lengths_and_primers(seed, n_genomes, len_lo, len_hi, n_pairs)
    seq, offsets = _alloc(lengths, out)
    _fill_genomes(seq, offsets, seed + 2, gcs, 0.005, 50)
    tmpls, planted = batched_templates(seed, lengths, fwd, rev)
    for g, off, t in tmpls:
        a = int(offsets[g]) + off
        seq[a:a + len(t)] = np.frombuffer(t, dtype=np.uint8)
    return Workload("batched", seq, offsets, np.arange(n_genomes, dtype=np.uint32), fwd, rev,
                    [i % 4 for i in range(n_pairs)], 3, 50, 2000, 0b1111, TmParams(min_tm=None), False, 0, 0,
                    planted, seed)


def dense(seed: int = SEED, n_genomes: int = 5000, median: float = 3.5e6, sigma: float = 0.4,
          out: Optional[np.ndarray] = None) -> Workload:
    """Dense-hit stress: tandem repeats in 30 % of genomes, 18-nt primers with 9 degenerate codes and
    k=4 (about 2 sites and 1 amplicon per kb of random sequence), window 50-5000, all orientations.
    Amplicons are counted and annotated with Tm; sequences are not extracted."""
    lengths, gcs = dense_layout(seed, n_genomes, median, sigma)
    seq, offsets = _alloc(lengths, out)
    _fill_genomes(seq, offsets, seed + 3, gcs, 0.005, 50)
    lib = _get_lib()
    for g, off, rlen, key, period in dense_repeats(seed, lengths):
        a = int(offsets[g])
        lib.synth_fill_tandem(seq.ctypes.data + a + off, rlen, key, period)
    fwd, rev = dense_primers(seed)
    return Workload("dense", seq, offsets, np.arange(n_genomes, dtype=np.uint32), fwd, rev, [DENSE_K], 3, 50, 5000,
                    0b1111, TmParams(min_tm=None), False, 0, 0, [], seed, False)


DENSE_K = 4   # mismatch budget of the dense workload: about 1 amplicon per kb of background


def dense_layout(seed: int, n_genomes: int, median: float, sigma: float):
    """Lengths and per-genome GC of the dense workload."""
    st_len = Stream(make_key(seed + 3, T_LEN, 0))
    lengths = [max(1000, int(round(median * math.exp(sigma * st_len.normal())))) for _ in range(n_genomes)]
    st_gc = Stream(make_key(seed + 3, T_GC, 0))
    gcs = [0.30 + 0.40 * st_gc.unit() for _ in range(n_genomes)]
    return lengths, gcs


def dense_repeats(seed: int, lengths: Sequence[int]):
    """The tandem repeats of the dense workload, in the order they are written: (genome, offset in the
    genome, length, key, period).  30 % of genomes carry 1-5 repeats of period 2-12, 1-20 kbp."""
    out = []
    for g, n in enumerate(lengths):
        st = Stream(make_key(seed + 3, T_TANDEM, g))
        if st.unit() >= 0.30:
            continue
        for r in range(st.randint(1, 5)):
            period = st.randint(2, 12)
            rlen = min(n, st.randint(1000, 20000))
            off = st.randint(0, max(0, n - rlen))
            out.append((g, off, rlen, make_key(seed + 3, T_TANDEM, g * 64 + r + 1), period))
    return out


def dense_primers(seed: int):
    pst = Stream(make_key(seed + 3, T_PRIMER, 0))
    fwd = [random_primer(pst, 18, 9, 3, codes="RYMKSWNNN")]
    rev = [random_primer(pst, 18, 9, 3, codes="RYMKSWNNN")]
    return fwd, rev


def random_small(seed: int, n_records: int, len_lo: int, len_hi: int, n_pairs: int = 1, plen_lo: int = 6,
                 plen_hi: int = 10, n_deg: int = 2, k_max: int = 2, clamp: int = 2, n_frac: float = 0.01,
                 alphabet: str = "ACGT", plant: int = 2, min_len: int = 10, max_len: int = 200,
                 fb: int = 4, rb: int = 5, trim: bool = True, codes: str = "RYMKSWNBDHV") -> Workload:
    """Tiny random workloads for brute-force pins and edge-case parity tests."""
    st = Stream(make_key(seed, 99, 0))
    lengths = [st.randint(len_lo, len_hi) for _ in range(n_records)]
    seq, offsets = _alloc(lengths, None)
    for g in range(n_records):
        a, b = int(offsets[g]), int(offsets[g + 1])
        for i in range(a, b):
            seq[i] = ord(st.choice(alphabet))
        if n_frac > 0:
            for i in range(a, b):
                if st.unit() < n_frac:
                    seq[i] = ord(st.choice("NRYnacgt"))
    fwd, rev, ks = [], [], []
    for _ in range(n_pairs):
        fwd.append(random_primer(st, st.randint(plen_lo, plen_hi), st.randint(0, n_deg), clamp, codes))
        rev.append(random_primer(st, st.randint(plen_lo, plen_hi), st.randint(0, n_deg), clamp, codes))
        ks.append(st.randint(0, k_max))
    planted: List[Planted] = []
    for g in range(n_records):
        if plant <= 0:
            break
        p = st.randint(0, n_pairs - 1)
        _plant(seq, offsets, g, st, plant, fwd[p], rev[p], p, lambda s: s.randint(0, 30), 1, planted)
    return Workload("random_small", seq, offsets, np.arange(n_records, dtype=np.uint32), fwd, rev, ks, clamp,
                    min_len, max_len, 0b1111, TmParams(min_tm=None), trim, fb, rb, planted, seed)


WORKLOADS = {"plain_small": plain_small, "plain_scale": plain_scale, "batched": batched, "dense": dense}


def serving_trace(seed: int, n_requests: int, rate_per_s: float, n_db_records: int, pairs_max: int = 32):
    """A Poisson request stream for the serving database: each request has 1-pairs_max degenerate
    pairs of 17-26 nt (0-6 codes), k of 0-3 per pair, and a genome subset that is a contiguous
    record range covering a log-uniform 1 %-100 % of the database."""
    st = Stream(make_key(seed + 5, T_SUBSET, 0))
    t, out = 0.0, []
    for _ in range(n_requests):
        t += -math.log(1.0 - st.unit()) / rate_per_s
        pairs = st.randint(1, pairs_max)
        fwd = [random_primer(st, st.randint(17, 26), st.randint(0, 6), 3) for _ in range(pairs)]
        rev = [random_primer(st, st.randint(17, 26), st.randint(0, 6), 3) for _ in range(pairs)]
        k = [st.randint(0, 3) for _ in range(pairs)]
        frac = math.exp(math.log(0.01) + (math.log(1.0) - math.log(0.01)) * st.unit())
        count = max(1, int(round(frac * n_db_records)))
        first = st.randint(0, n_db_records - count)
        out.append(dict(arrival=t, fwd=fwd, rev=rev, k=k, clamp=3, first_record=first, n_records=count, min_len=50,
                        max_len=2000, orient_mask=15))
    return out


def amplicon_reads(seed: int = SEED, n_reads: int = 2_000_000, read_len: int = 300, err: float = 0.01):
    """Amplicon-sequencing reads as FASTQ text (the input the paper's future-work FASTQ support is
    for): each read holds a concrete variant of the plain pair's forward primer 0-10 bases in, a
    random interior and the reverse complement of a variant of its reverse primer 0-10 bases before
    the end; a tenth of the reads are random; substitutions at rate `err`; qualities uniform on
    '!'..'J'.  Returns (FASTQ bytes as a uint8 array, the Workload of the same reads)."""
    pst = Stream(make_key(seed, T_PRIMER, 0))        # the plain pair
    fwd = random_primer(pst, 19, 2, 3)
    rev = random_primer(pst, 20, 3, 3)
    rng = np.random.default_rng(seed + 17)
    codes = np.frombuffer(b"ACGT", dtype=np.uint8)
    seqs = codes[rng.integers(0, 4, (n_reads, read_len))]
    vst = Stream(make_key(seed, T_PLANT, 0x5eed))
    fv = [np.frombuffer(concrete_variant(vst, fwd).encode(), dtype=np.uint8) for _ in range(32)]
    comp = bytes.maketrans(b"ACGT", b"TGCA")
    rv = [np.frombuffer(concrete_variant(vst, rev).encode().translate(comp)[::-1], dtype=np.uint8) for _ in range(32)]
    a = rng.integers(0, 11, n_reads)
    b = rng.integers(0, 11, n_reads)
    fi = rng.integers(0, 32, n_reads)
    ri = rng.integers(0, 32, n_reads)
    planted = rng.random(n_reads) >= 0.1
    gf = np.where(planted, a * 32 + fi, -1)
    gr = np.where(planted, b * 32 + ri, -1)
    for g in range(11 * 32):
        aa, k = divmod(g, 32)
        sel = np.nonzero(gf == g)[0]
        if len(sel):
            seqs[sel, aa:aa + len(fwd)] = fv[k]
        sel = np.nonzero(gr == g)[0]
        if len(sel):
            e = read_len - aa
            seqs[sel, e - len(rev):e] = rv[k]
    errs = rng.random((n_reads, read_len)) < err
    seqs[errs] = codes[rng.integers(0, 4, int(errs.sum()))]
    quals = rng.integers(33, 75, (n_reads, read_len), dtype=np.uint8)
    name_len = 10
    rec = 1 + name_len + 1 + read_len + 3 + read_len + 1
    text = np.empty((n_reads, rec), dtype=np.uint8)
    text[:, 0] = ord("@")
    idx = np.arange(n_reads)
    for d in range(name_len):
        text[:, 1 + d] = 48 + (idx // 10 ** (name_len - 1 - d)) % 10
    c = 1 + name_len
    text[:, c] = 10
    text[:, c + 1:c + 1 + read_len] = seqs
    c += 1 + read_len
    text[:, c:c + 3] = np.frombuffer(b"\n+\n", dtype=np.uint8)
    text[:, c + 3:c + 3 + read_len] = quals
    text[:, -1] = 10
    offsets = np.arange(n_reads + 1, dtype=np.int64) * read_len
    wl = Workload("amplicon_reads", seqs.reshape(-1), offsets, np.arange(n_reads, dtype=np.uint32), [fwd], [rev], [2],
                  3, 50, 2000, 0b1111, TmParams(min_tm=None), True, 0, 0, [], seed)
    return text.reshape(-1), wl
