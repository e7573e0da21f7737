"""Device-side drawing of large synthetic workloads (batched, serving database).

The genomes come out byte-identical to the host generator's for the same seed: bases use the same
counter-based draws, runs of N are computed by the same C routine on the host and written on the
device, and planted templates are built on the host and scattered.  Device memory is a torch
uint8 tensor; nothing here touches the in-silico PCR arithmetic.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

from . import (SEED, T_GC, T_LEN, T_NRUN, T_BASES, Planted, Stream, TmParams, Workload, _get_lib, batched_lengths_and_primers,
               DENSE_K, batched_templates, dense_layout, dense_primers, dense_repeats, make_key)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "_synth_gpu.cu")
_LIB = os.path.join(_HERE, "_synth_gpu.so")
_lib = None
_lock = threading.Lock()

FILL_ITEM = np.dtype([("out_off", "<u8"), ("first", "<u8"), ("count", "<u8"), ("key", "<u8"), ("gc", "<f8")])


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC",
                               "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            vp, u64 = ctypes.c_void_p, ctypes.c_uint64
            L.synth_gpu_fill.argtypes = [vp, vp, u64, vp]
            L.synth_gpu_runs.argtypes = [vp, vp, vp, u64, vp]
            L.synth_gpu_scatter.argtypes = [vp, vp, vp, vp, u64, vp]
            for f in (L.synth_gpu_fill, L.synth_gpu_runs, L.synth_gpu_scatter):
                f.restype = ctypes.c_int
            _lib = L
    return _lib


@dataclass
class DeviceWorkload:
    """A workload whose genomes live in device memory (d_seq: torch uint8 tensor)."""
    name: str
    d_seq: object
    offsets: np.ndarray
    genome_ids: np.ndarray
    fwd: List[str]
    rev: List[str]
    k: List[int]
    clamp: int
    min_len: int
    max_len: int
    orient_mask: int
    tm: TmParams
    trim: bool
    fb_len: int
    rb_len: int
    planted: List[Planted] = field(default_factory=list)
    seed: int = SEED
    extract: bool = True

    @property
    def n_records(self) -> int:
        return len(self.offsets) - 1

    @property
    def total_bp(self) -> int:
        return int(self.offsets[-1])

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def host_subset(self, records: Sequence[int]) -> Workload:
        """The given records copied to the host as an ordinary Workload (for oracle samples)."""
        recs = list(records)
        lens = [int(self.offsets[i + 1] - self.offsets[i]) for i in recs]
        offs = np.zeros(len(recs) + 1, dtype=np.int64)
        offs[1:] = np.cumsum(lens)
        seq = np.empty(int(offs[-1]), dtype=np.uint8)
        for j, i in enumerate(recs):
            seq[offs[j]:offs[j + 1]] = self.d_seq[int(self.offsets[i]):int(self.offsets[i + 1])].cpu().numpy()
        return Workload(self.name + "-subset", seq, offs, self.genome_ids[recs].copy(), list(self.fwd), list(self.rev),
                        list(self.k), self.clamp, self.min_len, self.max_len, self.orient_mask, self.tm, self.trim,
                        self.fb_len, self.rb_len, [], self.seed, self.extract)

    subset = host_subset


def draw_genomes(seed_tag: int, lengths: Sequence[int], gcs: Sequence[float], n_frac: float = 0.005,
                 run_max: int = 50, device: str = "cuda", chunk: int = 1 << 26, genome_first: int = 0):
    """Genomes drawn on the device exactly as synth._fill_genomes draws them on the host.  lengths
    and gcs describe genomes genome_first, genome_first + 1, ... (their keys use those indices)."""
    import torch

    L = _get()
    lib = _get_lib()
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(np.asarray(lengths, dtype=np.int64))
    d = torch.empty(int(offsets[-1]), dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream().cuda_stream
    items = []
    for g, n in enumerate(lengths):
        key = make_key(seed_tag, T_BASES, genome_first + g)
        for a in range(0, n, chunk):
            items.append((int(offsets[g]) + a, a, min(chunk, n - a), key, float(gcs[g])))
    arr = np.array(items, dtype=FILL_ITEM)
    torch.cuda.synchronize()
    if len(arr):
        rc = L.synth_gpu_fill(d.data_ptr(), arr.ctypes.data, len(arr), stream)
        if rc:
            raise RuntimeError(f"device fill failed ({rc})")
    if n_frac > 0:
        starts, lens_ = [], []
        for g, n in enumerate(lengths):
            key = make_key(seed_tag, T_NRUN, genome_first + g)
            cnt = lib.synth_nrun_list(n, key, n_frac, run_max, None, None, 0)
            st = np.empty(cnt, dtype=np.uint64)
            ln = np.empty(cnt, dtype=np.uint32)
            lib.synth_nrun_list(n, key, n_frac, run_max, st.ctypes.data, ln.ctypes.data, cnt)
            starts.append(st + np.uint64(offsets[g]))
            lens_.append(ln)
        st = torch.from_numpy(np.concatenate(starts)).to(device)
        ln = torch.from_numpy(np.concatenate(lens_)).to(device)
        rc = L.synth_gpu_runs(d.data_ptr(), st.data_ptr(), ln.data_ptr(), len(st), stream)
        torch.cuda.synchronize()
        if rc:
            raise RuntimeError(f"device N runs failed ({rc})")
    return d, offsets


def scatter(d, offsets, tmpls) -> None:
    """Write host-built templates (genome, offset, bytes) into the device genomes."""
    import torch

    if not tmpls:
        return
    src = np.frombuffer(b"".join(t for _, _, t in tmpls), dtype=np.uint8)
    src_off = np.zeros(len(tmpls) + 1, dtype=np.uint64)
    src_off[1:] = np.cumsum([len(t) for _, _, t in tmpls])
    dst = np.array([int(offsets[g]) + o for g, o, _ in tmpls], dtype=np.uint64)
    ds, do, dd = (torch.from_numpy(x).cuda() for x in (src.copy(), src_off, dst))
    rc = _get().synth_gpu_scatter(d.data_ptr(), ds.data_ptr(), do.data_ptr(), dd.data_ptr(), len(tmpls),
                                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    if rc:
        raise RuntimeError(f"device scatter failed ({rc})")


def batched(seed: int = SEED, n_genomes: int = 50_000, len_lo: float = 1e4, len_hi: float = 1.2e7,
            n_pairs: int = 8) -> DeviceWorkload:
    """synth.batched drawn on the device (byte-identical)."""
    lengths, gcs, fwd, rev = batched_lengths_and_primers(seed, n_genomes, len_lo, len_hi, n_pairs)
    d, offsets = draw_genomes(seed + 2, lengths, gcs)
    tmpls, planted = batched_templates(seed, lengths, fwd, rev)
    scatter(d, offsets, tmpls)
    return DeviceWorkload("batched", d, offsets, np.arange(n_genomes, dtype=np.uint32), fwd, rev,
                          [i % 4 for i in range(n_pairs)], 3, 50, 2000, 0b1111, TmParams(min_tm=None), False, 0, 0,
                          planted, seed)


def dense(seed: int = SEED, n_genomes: int = 5000, median: float = 3.5e6, sigma: float = 0.4) -> DeviceWorkload:
    """synth.dense drawn on the device (byte-identical).  The tandem repeats are written on the host
    in their order; repeats that overlap within a genome are merged into one template first, so the
    device writes disjoint templates and later repeats win exactly as on the host."""
    lengths, gcs = dense_layout(seed, n_genomes, median, sigma)
    d, offsets = draw_genomes(seed + 3, lengths, gcs)
    lib = _get_lib()
    by_genome = {}
    for rep in dense_repeats(seed, lengths):
        by_genome.setdefault(rep[0], []).append(rep)
    tmpls = []
    for g, reps in by_genome.items():
        # groups of repeats whose spans overlap (transitively), each group written in repeat order
        spans = sorted(range(len(reps)), key=lambda i: reps[i][1])
        groups, cur, cur_end = [], [], -1
        for i in spans:
            a, n = reps[i][1], reps[i][2]
            if cur and a < cur_end:
                cur.append(i)
                cur_end = max(cur_end, a + n)
            else:
                if cur:
                    groups.append(cur)
                cur, cur_end = [i], a + n
        if cur:
            groups.append(cur)
        for grp in groups:
            lo = min(reps[i][1] for i in grp)
            hi = max(reps[i][1] + reps[i][2] for i in grp)
            buf = np.zeros(hi - lo, dtype=np.uint8)
            for i in sorted(grp):
                _, off, rlen, key, period = reps[i]
                lib.synth_fill_tandem(buf.ctypes.data + (off - lo), rlen, key, period)
            tmpls.append((g, lo, buf.tobytes()))
    scatter(d, offsets, tmpls)
    fwd, rev = dense_primers(seed)
    return DeviceWorkload("dense", d, offsets, np.arange(n_genomes, dtype=np.uint32), fwd, rev, [DENSE_K], 3, 50, 5000,
                          0b1111, TmParams(min_tm=None), False, 0, 0, [], seed, False)


def serving_layout(seed: int = SEED, n_genomes: int = 40_000, median: float = 3.5e6, sigma: float = 0.4):
    """Lengths and per-genome GC of the serving database (plain_scale distributions)."""
    st_len = Stream(make_key(seed + 4, T_LEN, 0))
    lengths = [max(1000, int(round(median * math.exp(sigma * st_len.normal())))) for _ in range(n_genomes)]
    st_gc = Stream(make_key(seed + 4, T_GC, 0))
    gcs = [0.30 + 0.40 * st_gc.unit() for _ in range(n_genomes)]
    return lengths, gcs


def serving_db(seed: int = SEED, n_genomes: int = 40_000, median: float = 3.5e6, sigma: float = 0.4) -> DeviceWorkload:
    """Serving database: lognormal lengths and per-genome GC as plain_scale, 0.5 % N, no planting."""
    lengths, gcs = serving_layout(seed, n_genomes, median, sigma)
    d, offsets = draw_genomes(seed + 4, lengths, gcs)
    return DeviceWorkload("serving_db", d, offsets, np.arange(n_genomes, dtype=np.uint32), [], [], [], 3, 50, 2000,
                          15, TmParams(min_tm=None), False, 0, 0, [], seed)


def serving_db_chunks(seed: int = SEED, n_genomes: int = 40_000, median: float = 3.5e6, sigma: float = 0.4,
                      chunk_bases: int = 12 << 30):
    """The serving database drawn in genome ranges of about chunk_bases: yields (first genome, device
    ASCII tensor, offsets from 0) so a caller can pack each range and release it."""
    lengths, gcs = serving_layout(seed, n_genomes, median, sigma)
    a = 0
    while a < n_genomes:
        b, acc = a, 0
        while b < n_genomes and (acc == 0 or acc + lengths[b] <= chunk_bases):
            acc += lengths[b]
            b += 1
        d, offs = draw_genomes(seed + 4, lengths[a:b], gcs[a:b], genome_first=a)
        yield a, d, offs
        del d
        a = b
