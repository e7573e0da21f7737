"""ORACLE -- TEST INFRASTRUCTURE ONLY.

Plain, slow CPU restatement of the AmpliconHunter2 in-silico PCR path (arXiv 2511.00170),
written in C (``oracle.c``) and wrapped here with ctypes.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this package; the
product path never does.  It shares no code, tables or helpers with the CUDA path.

Functions follow the paper's passages (see the header of ``oracle.c`` for the readings R1-R16):

* :func:`scan`    -- Supplementary, "Primer matching and clamp logic".
* :func:`pair`    -- Supplementary, "Amplicon calling and orientation".
* :func:`tm_hits` -- Section "Implementations" (AHv2 Tm_NN) and "Primer degeneracy".
* :func:`extract` -- Supplementary, "Primer trimming and barcode extraction", "Headers and outputs".

Parity of the nearest-neighbour parameter tables against Biopython is unpinned (neither the
publications nor Biopython are available here); the arithmetic is pinned by the tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None
_lock = threading.Lock()

HIT_DTYPE = np.dtype([("record", "<u4"), ("pos", "<u4"), ("pair", "<u2"), ("primer", "u1"),
                      ("strand", "u1"), ("mism", "u1"), ("pad", "u1", 3)])
AMP_DTYPE = np.dtype([("record", "<u4"), ("pair", "<u4"), ("start", "<u4"), ("end", "<u4"),
                      ("hit_i", "<u4"), ("hit_j", "<u4"), ("orient", "u1"), ("pad", "u1", 3)])
ORIENT_NAMES = ("FR", "RF", "FF", "RR")


class _TmParams(ctypes.Structure):
    _fields_ = [("Na", ctypes.c_double), ("K", ctypes.c_double), ("Tris", ctypes.c_double),
                ("Mg", ctypes.c_double), ("dNTPs", ctypes.c_double), ("dnac1", ctypes.c_double),
                ("dnac2", ctypes.c_double), ("saltcorr", ctypes.c_int), ("selfcomp", ctypes.c_int),
                ("variants", ctypes.c_int), ("nn_table", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, gcc) next to this file."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            vp, i64, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32
            L.or_check_primer.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_int]
            L.or_check_primer.restype = ctypes.c_int
            L.or_scan.argtypes = [vp, vp, u32, u32, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
            L.or_scan.restype = i64
            L.or_pair.argtypes = [vp, i64, vp, vp, u32, u32, u32, ctypes.POINTER(vp)]
            L.or_pair.restype = i64
            L.or_duplex_sums.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            L.or_duplex_sums.restype = ctypes.c_int
            L.or_duplex_sums_set.argtypes = [ctypes.c_int, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            L.or_duplex_sums_set.restype = ctypes.c_int
            L.or_tm_duplex.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int,
                                       ctypes.POINTER(_TmParams), ctypes.POINTER(ctypes.c_int)]
            L.or_tm_duplex.restype = ctypes.c_double
            L.or_tm_site.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(_TmParams), ctypes.POINTER(ctypes.c_int)]
            L.or_tm_site.restype = ctypes.c_double
            L.or_tm_hits.argtypes = [vp, vp, vp, i64, vp, vp, vp, ctypes.c_int, ctypes.POINTER(_TmParams), vp, vp]
            L.or_tm_hits.restype = None
            L.or_extract.argtypes = [vp, vp, vp, vp, i64, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
            L.or_extract.restype = i64
            L.or_free.argtypes = [vp]
            L.or_free.restype = None
            L.or_nn_entry.argtypes = [ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
            L.or_nn_entry.restype = ctypes.c_int
            L.or_nn_entry_set.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
            L.or_nn_entry_set.restype = ctypes.c_int
            L.or_free_mg.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_free_mg.restype = ctypes.c_double
            _lib = L
    return _lib


def _params(tm) -> _TmParams:
    return _TmParams(float(tm.Na), float(tm.K), float(tm.Tris), float(tm.Mg), float(tm.dNTPs), float(tm.dnac1),
                     float(tm.dnac2), int(tm.saltcorr), int(getattr(tm, "selfcomp", 0)),
                     int(getattr(tm, "variants", 0)), int(getattr(tm, "nn_table", 0)))


def _strs(xs: Sequence[str]):
    arr = (ctypes.c_char_p * len(xs))(*[x.encode("ascii") for x in xs])
    return arr


def check_primer(p: str, clamp: int, k: int) -> int:
    return _get().or_check_primer(p.encode("ascii"), clamp, k)


# ------------------------------------------------------------------------------------------ scan
def scan(wl, threads: int = 0) -> np.ndarray:
    """All hits sorted by (record, pair, pos, strand, primer); dtype :data:`HIT_DTYPE`."""
    L = _get()
    seq = np.ascontiguousarray(wl.seq, dtype=np.uint8)
    offs = np.ascontiguousarray(wl.offsets, dtype=np.int64)
    ks = np.ascontiguousarray(np.asarray(wl.k, dtype=np.uint8))
    fw, rv = _strs(wl.fwd), _strs(wl.rev)
    out = ctypes.c_void_p()
    threads = threads or (os.cpu_count() or 1)
    n = L.or_scan(seq.ctypes.data, offs.ctypes.data, wl.n_records, len(wl.fwd), ctypes.cast(fw, ctypes.c_void_p),
                  ctypes.cast(rv, ctypes.c_void_p), ks.ctypes.data, int(wl.clamp), int(threads), ctypes.byref(out))
    res = np.empty(n, dtype=HIT_DTYPE)
    if n:
        ctypes.memmove(res.ctypes.data, out.value, n * HIT_DTYPE.itemsize)
    L.or_free(out)
    return res


def primer_lengths(wl) -> Tuple[np.ndarray, np.ndarray]:
    return (np.array([len(p) for p in wl.fwd], dtype=np.uint32), np.array([len(p) for p in wl.rev], dtype=np.uint32))


# ------------------------------------------------------------------------------------------ pair
def pair(wl, hits: np.ndarray, orient_mask: Optional[int] = None) -> np.ndarray:
    L = _get()
    lf, lr = primer_lengths(wl)
    hits = np.ascontiguousarray(hits, dtype=HIT_DTYPE)
    out = ctypes.c_void_p()
    mask = wl.orient_mask if orient_mask is None else orient_mask
    n = L.or_pair(hits.ctypes.data, len(hits), lf.ctypes.data, lr.ctypes.data, int(wl.min_len), int(wl.max_len),
                  int(mask), ctypes.byref(out))
    res = np.empty(n, dtype=AMP_DTYPE)
    if n:
        ctypes.memmove(res.ctypes.data, out.value, n * AMP_DTYPE.itemsize)
    L.or_free(out)
    return res


# ------------------------------------------------------------------------------------------ Tm
def duplex_sums(seq: str, cseq: str, nn_table: int = 0) -> Optional[Tuple[float, float]]:
    """(dH kcal/mol, dS cal/(K mol)) before salt and concentration terms, or None if undefined."""
    dh, ds = ctypes.c_double(), ctypes.c_double()
    ok = _get().or_duplex_sums_set(nn_table, seq.encode(), cseq.encode(), len(seq), ctypes.byref(dh),
                                   ctypes.byref(ds))
    return (dh.value, ds.value) if ok else None


NN_WC, NN_INTERNAL, NN_TERMINAL, NN_SCALAR = range(4)


# nearest-neighbour sets, Biopython's numbering (6 and 7, RNA_NN2 and RNA_NN3, are not built)
NN_SETS = {0: "DNA_NN3", 1: "DNA_NN1", 2: "DNA_NN2", 3: "DNA_NN3", 4: "DNA_NN4", 5: "RNA_NN1", 8: "R_DNA_NN1"}


def nn_entry(table: int, key: str, nn_table: int = 0) -> Optional[Tuple[float, float]]:
    """One stored parameter (dH, dS) as written in the oracle's tables, or None (for pins only);
    table NN_WC and NN_SCALAR read set nn_table."""
    dh, ds = ctypes.c_double(), ctypes.c_double()
    ok = _get().or_nn_entry_set(nn_table, table, key.encode(), ctypes.byref(dh), ctypes.byref(ds))
    return (dh.value, ds.value) if ok else None


def tm_duplex(seq: str, cseq: str, tm) -> Optional[float]:
    d = ctypes.c_int()
    p = _params(tm)
    t = _get().or_tm_duplex(seq.encode(), cseq.encode(), len(seq), ctypes.byref(p), ctypes.byref(d))
    return t if d.value else None


def parse_fasta(text: bytes) -> Tuple[List[str], List[bytes]]:
    """FASTA records, line by line (Abstract: the input is FASTA): a line starting with '>' opens a
    record named by the rest of the line (a trailing '\\r' dropped); every other line adds its bytes
    except '\\r', ' ' and '\\t' to the open record; lines before the first header are ignored."""
    names, seqs = [], []
    for line in text.split(b"\n"):
        if line.startswith(b">"):
            names.append(line[1:].rstrip(b"\r").decode("latin-1"))
            seqs.append(bytearray())
        elif seqs:
            seqs[-1] += bytes(c for c in line if c not in b"\r \t")
    return names, [bytes(s) for s in seqs]


def amplicon_fasta(records, names: Sequence[str], sources: Optional[Sequence[str]], barcodes: bool) -> bytes:
    """FASTA text of amplicons with the headers of Supplementary "Headers and outputs": records are
    (record, start, end, orient, tm, (amplicon, fb, rb, site i, site j)); the id is the record name
    up to its first blank; coordinates 1-based inclusive; Tm to two decimals (NA if undefined); the
    forward primer's site is site j for RF, site i otherwise; barcodes only when requested."""
    out = []
    for rec, start, end, orient, tm, f in records:
        name = names[rec]
        for i, ch in enumerate(name):
            if ch in " \t":
                name = name[:i]
                break
        h = ">" + name
        if sources is not None and sources[rec] is not None:
            h += ".source=" + sources[rec]
        h += ".coordinates=%d-%d" % (start + 1, end)
        h += ".Tm=" + ("NA" if tm != tm else "%.2f" % tm)
        h += ".orientation=" + ORIENT_NAMES[orient]
        fp, rp = (f[4], f[3]) if orient == 1 else (f[3], f[4])
        h += ".fprimer=" + fp.decode("latin-1") + ".rprimer=" + rp.decode("latin-1")
        if barcodes:
            h += ".fb=" + f[1].decode("latin-1") + ".rb=" + f[2].decode("latin-1")
        out.append(h.encode("latin-1") + b"\n" + f[0] + b"\n")
    return b"".join(out)


def parse_fastq(text: bytes) -> Tuple[List[str], List[bytes], List[bytes]]:
    """FASTQ records of four lines ('@' name, bases, '+', qualities; '\\r' dropped; empty lines after
    the last record ignored): names, bases, qualities."""
    lines = [ln.replace(b"\r", b"") for ln in text.split(b"\n")]
    while lines and lines[-1] == b"":
        lines.pop()
    names, seqs, quals = [], [], []
    for r in range(0, len(lines), 4):
        head = lines[r]
        assert head.startswith(b"@"), "not FASTQ"
        names.append(head[1:].decode("latin-1"))
        seqs.append(lines[r + 1] if r + 1 < len(lines) else b"")
        quals.append(lines[r + 3] if r + 3 < len(lines) else b"")
        assert len(seqs[-1]) == len(quals[-1]), "qualities differ in length from the bases"
    return names, seqs, quals


def amplicon_qualities(wl, hits: np.ndarray, amps: np.ndarray, quals: Sequence[bytes]) -> List[bytes]:
    """Per amplicon the qualities of its sequence field (Supplementary "Primer trimming and barcode
    extraction"): the bases from site i's start to site j's end, or with trimming from site i's end
    to site j's start (empty if they overlap), reversed for RF as the bases are (qualities are not
    complemented)."""
    lf, lr = primer_lengths(wl)
    out = []
    for a in amps:
        hi, hj = hits[a["hit_i"]], hits[a["hit_j"]]
        li = (lf if hi["primer"] == 0 else lr)[hi["pair"]]
        lj = (lf if hj["primer"] == 0 else lr)[hj["pair"]]
        s_i, e_i, s_j, e_j = int(hi["pos"]), int(hi["pos"]) + int(li), int(hj["pos"]), int(hj["pos"]) + int(lj)
        lo, hi_ = (e_i, max(e_i, s_j)) if wl.trim else (s_i, e_j)
        q = quals[int(a["record"])][lo:hi_]
        out.append(q[::-1] if int(a["orient"]) == 1 else q)
    return out


def amplicon_fastq(records, names: Sequence[str], sources: Optional[Sequence[str]], barcodes: bool) -> bytes:
    """FASTQ text: records are (record, start, end, orient, tm, fields, qualities); the header as in
    amplicon_fasta with '@', then the sequence, '+' and the qualities."""
    out = []
    for rec in records:
        fa = amplicon_fasta([rec[:6]], names, sources, barcodes)
        out.append(b"@" + fa[1:] + b"+\n" + rec[6] + b"\n")
    return b"".join(out)


def free_mg(mg_mM: float, dntps_mM: float) -> float:
    """Free Mg2+ (mM) beside dNTPs that bind it one to one (salt method 7's input)."""
    return _get().or_free_mg(float(mg_mM), float(dntps_mM))


def tm_site(primer: str, site: str, tm, k: Optional[int] = None, clamp: int = 0) -> Optional[float]:
    """Tm of `primer` at `site` (site bases in the primer's 5'->3' orientation): the maximum over the
    primer's concrete variants with at most `k` mismatches to the site (default: any number) and an
    exact match over the last `clamp` positions (reading R14); None when no such variant is defined."""
    st = ctypes.c_int()
    p = _params(tm)
    k = len(primer) if k is None else k
    t = _get().or_tm_site(primer.encode(), site.encode(), len(primer), int(k), int(clamp), ctypes.byref(p),
                          ctypes.byref(st))
    return None if st.value else t


def tm_hits(wl, hits: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Per hit: Tm (max over the primer's concrete variants; with ``wl.tm.variants == 1`` only those
    that match the site within the pair's k and the clamp) and status (0 ok, 1 undefined)."""
    L = _get()
    hits = np.ascontiguousarray(hits, dtype=HIT_DTYPE)
    seq = np.ascontiguousarray(wl.seq, dtype=np.uint8)
    offs = np.ascontiguousarray(wl.offsets, dtype=np.int64)
    tm = np.empty(len(hits), dtype=np.float64)
    st = np.empty(len(hits), dtype=np.uint8)
    fw, rv = _strs(wl.fwd), _strs(wl.rev)
    p = _params(wl.tm)
    ks = np.ascontiguousarray(np.asarray(wl.k, dtype=np.uint8))
    L.or_tm_hits(seq.ctypes.data, offs.ctypes.data, hits.ctypes.data, len(hits), ctypes.cast(fw, ctypes.c_void_p),
                 ctypes.cast(rv, ctypes.c_void_p), ks.ctypes.data, int(wl.clamp), ctypes.byref(p), tm.ctypes.data,
                 st.ctypes.data)
    return tm, st


def amplicon_tm(amps: np.ndarray, hit_tm: np.ndarray, hit_status: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Amplicon Tm = the lower of its two site Tms (reading R13); status 1 if either is undefined."""
    ti, tj = hit_tm[amps["hit_i"]], hit_tm[amps["hit_j"]]
    si, sj = hit_status[amps["hit_i"]], hit_status[amps["hit_j"]]
    status = ((si != 0) | (sj != 0)).astype(np.uint8)
    tm = np.where(status == 0, np.minimum(ti, tj), np.nan)
    return tm, status


def tm_keep(tm: np.ndarray, status: np.ndarray, min_tm: Optional[float]) -> np.ndarray:
    """Filter: keep iff defined and Tm >= min_tm (no filter: keep all) (readings R15, R16)."""
    if min_tm is None:
        return np.ones(len(tm), dtype=bool)
    with np.errstate(invalid="ignore"):
        return (status == 0) & (tm >= min_tm)


# Two FP64 evaluations of the same Tm may differ in their last digits (summation order, libm), and
# the engine's Tm is held to within this distance of the oracle's; a decision closer to the
# threshold than this is flagged rather than trusted (reading R16: the filter compares unrounded
# values).
NEAR_TOL = 1e-9


def tm_near(tm: np.ndarray, status: np.ndarray, min_tm: Optional[float]) -> np.ndarray:
    """Near-threshold flag: Tm defined and within NEAR_TOL degrees of min_tm (never without one)."""
    if min_tm is None:
        return np.zeros(len(tm), dtype=bool)
    with np.errstate(invalid="ignore"):
        return (status == 0) & (np.abs(tm - min_tm) <= NEAR_TOL)


# ------------------------------------------------------------------------------------------ extract
def extract(wl, hits: np.ndarray, amps: np.ndarray, trim: Optional[bool] = None, fb: Optional[int] = None,
            rb: Optional[int] = None) -> List[Tuple[str, str, str, str, str]]:
    """Per amplicon: (sequence, forward barcode, reverse barcode, site i bases, site j bases)."""
    L = _get()
    lf, lr = primer_lengths(wl)
    trim = wl.trim if trim is None else trim
    fb = wl.fb_len if fb is None else fb
    rb = wl.rb_len if rb is None else rb
    seq = np.ascontiguousarray(wl.seq, dtype=np.uint8)
    offs = np.ascontiguousarray(wl.offsets, dtype=np.int64)
    hits = np.ascontiguousarray(hits, dtype=HIT_DTYPE)
    amps = np.ascontiguousarray(amps, dtype=AMP_DTYPE)
    fo = np.zeros(5 * len(amps) + 1, dtype=np.int64)
    total = L.or_extract(seq.ctypes.data, offs.ctypes.data, hits.ctypes.data, amps.ctypes.data, len(amps),
                         lf.ctypes.data, lr.ctypes.data, int(trim), int(fb), int(rb), None, fo.ctypes.data)
    arena = ctypes.create_string_buffer(max(1, total))
    L.or_extract(seq.ctypes.data, offs.ctypes.data, hits.ctypes.data, amps.ctypes.data, len(amps), lf.ctypes.data,
                 lr.ctypes.data, int(trim), int(fb), int(rb), arena, fo.ctypes.data)
    raw = arena.raw[:total].decode("ascii")
    out = []
    for m in range(len(amps)):
        f = [raw[fo[5 * m + q]:fo[5 * m + q + 1]] for q in range(5)]
        out.append(tuple(f))
    return out


# ------------------------------------------------------------------------------------------ all
@dataclass
class Result:
    hits: np.ndarray
    amps: np.ndarray          # all paired amplicons (orientation-filtered), before the Tm filter
    hit_tm: np.ndarray
    hit_status: np.ndarray
    amp_tm: np.ndarray
    amp_status: np.ndarray
    keep: np.ndarray
    seqs: Optional[List[Tuple[str, str, str, str, str]]]   # for the kept amplicons, in order
    near: Optional[np.ndarray] = None    # Tm within NEAR_TOL of min_tm
    min_tm: Optional[float] = None       # the threshold the filter used (None: no filter)


def run(wl, threads: int = 0, with_seqs: bool = True) -> Result:
    hits = scan(wl, threads)
    amps = pair(wl, hits)
    htm, hst = tm_hits(wl, hits)
    atm, ast = amplicon_tm(amps, htm, hst)
    keep = tm_keep(atm, ast, wl.tm.min_tm)
    seqs = extract(wl, hits, amps[keep]) if with_seqs else None
    return Result(hits, amps, htm, hst, atm, ast, keep, seqs, tm_near(atm, ast, wl.tm.min_tm), wl.tm.min_tm)
