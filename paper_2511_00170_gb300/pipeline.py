"""The whole in-silico PCR path through the C ABI: pack -> scan -> pair -> Tm -> extract.

Sequencing of C calls only; every step runs in libah.so.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Tuple

import numpy as np

from . import ah


@dataclass
class Params:
    fwd: List[str]
    rev: List[str]
    k: List[int]
    clamp: int
    min_len: int
    max_len: int
    orient_mask: int = 15
    Na: float = 50.0
    K: float = 0.0
    Tris: float = 0.0
    Mg: float = 0.0
    dNTPs: float = 0.0
    dnac1: float = 25.0
    dnac2: float = 25.0
    saltcorr: int = 5
    min_tm: Optional[float] = None
    trim: bool = False
    fb_len: int = 0
    rb_len: int = 0
    variants: int = 0
    selfcomp: int = 0
    filter: Optional[bool] = None   # None: filter iff min_tm is set; False: annotate the decision only
    nn_table: int = 0               # nearest-neighbour set (Biopython's numbering; 0 the default DNA_NN3)

    @classmethod
    def from_workload(cls, wl) -> "Params":
        t = wl.tm
        return cls(list(wl.fwd), list(wl.rev), list(wl.k), wl.clamp, wl.min_len, wl.max_len, wl.orient_mask, t.Na, t.K,
                   t.Tris, t.Mg, t.dNTPs, t.dnac1, t.dnac2, t.saltcorr, t.min_tm, wl.trim, wl.fb_len, wl.rb_len,
                   getattr(t, "variants", 0), getattr(t, "selfcomp", 0), None, getattr(t, "nn_table", 0))

    def tm_params(self) -> ah.ah_tm_params:
        return ah.tm_params(self.Na, self.K, self.Tris, self.Mg, self.dNTPs, self.dnac1, self.dnac2, self.saltcorr,
                            self.min_tm, self.variants, self.selfcomp, self.filter, self.nn_table)


@dataclass
class Output:
    hits: np.ndarray            # ah.HIT_DTYPE
    amps: np.ndarray            # ah.AMP_DTYPE (after the Tm filter when one is set)
    arena: Optional[bytes]
    field_off: Optional[np.ndarray]

    def fields(self, m: int) -> Tuple[str, str, str, str, str]:
        o = self.field_off
        return tuple(self.arena[int(o[5 * m + f]):int(o[5 * m + f + 1])].decode("ascii") for f in range(5))


class Engine:
    """Owns a context and, per run, the device objects of one step."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        self.ctx = ah.ah_ctx_create(device, stream)
        self._primers = None
        self._pkey = None

    def close(self):
        if self._primers is not None:
            ah.ah_primers_free(self._primers)
            self._primers = None
        if self.ctx is not None:
            ah.ah_ctx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def primers(self, p: Params):
        key = (tuple(p.fwd), tuple(p.rev), tuple(p.k), p.clamp)
        if key != self._pkey:
            if self._primers is not None:
                ah.ah_primers_free(self._primers)
            self._primers = ah.ah_primers_create(self.ctx, p.fwd, p.rev, p.k, p.clamp)
            self._pkey = key
        return self._primers

    def pack(self, seq: np.ndarray, offsets: np.ndarray, genome_ids=None):
        return ah.ah_pack_batch(self.ctx, seq, offsets, genome_ids)

    def pack_device(self, d_seq: int, offsets: np.ndarray, genome_ids=None):
        return ah.ah_pack_batch_device(self.ctx, d_seq, offsets, genome_ids)

    def step(self, batch, p: Params, with_seqs: bool = True, copy_out: bool = True):
        """One pass of the path over a packed batch.  Returns Output (host copies) or, with
        copy_out=False, the device objects (hits, amps) for the caller to free."""
        pr = self.primers(p)
        hits = ah.ah_scan_primers(self.ctx, batch, pr)
        amps = ah.ah_pair_amplicons(self.ctx, batch, pr, hits, p.min_len, p.max_len, p.orient_mask)
        ah.ah_tm_filter(self.ctx, batch, pr, hits, amps, p.tm_params())
        if with_seqs:
            ah.ah_extract_barcodes(self.ctx, batch, pr, hits, amps, p.trim, p.fb_len, p.rb_len)
        if not copy_out:
            return hits, amps
        try:
            ah.ah_ctx_synchronize(self.ctx)
            h = ah.ah_hits_copy(hits)
            a = ah.ah_amplicons_copy(amps)
            arena, off = ah.ah_amplicons_seq_copy(amps) if with_seqs else (None, None)
            return Output(h, a, arena, off)
        finally:
            ah.ah_hits_free(hits)
            ah.ah_amplicons_free(amps)

    def plan(self, batch, p: Params, with_seqs: bool = True, autotune: bool = False, persistent: int = -1, **caps):
        """A graph-captured plan of the whole step over `batch` (see ah_plan_create)."""
        prm = ah.plan_params(p.min_len, p.max_len, p.orient_mask, p.tm_params(), with_seqs, p.trim, p.fb_len, p.rb_len,
                             autotune, persistent, **caps)
        return ah.ah_plan_create(self.ctx, batch, self.primers(p), prm)

    def plan_output(self, plan, with_seqs: bool = True) -> Output:
        hits, amps = ah.ah_plan_results(plan, self.ctx)
        try:
            h = ah.ah_hits_copy(hits)
            a = ah.ah_amplicons_copy(amps)
            arena, off = ah.ah_amplicons_seq_copy(amps) if with_seqs else (None, None)
            return Output(h, a, arena, off)
        finally:
            ah.ah_hits_free(hits)
            ah.ah_amplicons_free(amps)

    def run_workload(self, wl, with_seqs: bool = True) -> Output:
        batch = self.pack(wl.seq, wl.offsets, wl.genome_ids)
        try:
            return self.step(batch, Params.from_workload(wl), with_seqs)
        finally:
            ah.ah_batch_free(batch)
