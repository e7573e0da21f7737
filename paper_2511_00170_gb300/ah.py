"""ctypes binding of the engine's C ABI (``include/ah.h``).

Argument marshalling only: every function has the name of the C entry point it calls, converts
Python/numpy arguments to plain pointers and sizes, raises :class:`AhError` on a non-OK status,
and returns handles or numpy arrays.  All computation happens in ``libah.so``.  There is no
fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libah.so")

AH_OK, AH_EINVAL, AH_ENOMEM, AH_ECUDA, AH_EOVERFLOW, AH_ETIMEOUT, AH_EJIT, AH_EINTERNAL, AH_ELIMIT, AH_ECANCELED = range(10)
STATUS_NAMES = {0: "AH_OK", 1: "AH_EINVAL", 2: "AH_ENOMEM", 3: "AH_ECUDA", 4: "AH_EOVERFLOW", 5: "AH_ETIMEOUT",
                6: "AH_EJIT", 7: "AH_EINTERNAL", 8: "AH_ELIMIT", 9: "AH_ECANCELED"}
AH_FR, AH_RF, AH_FF, AH_RR = 1, 2, 4, 8

HIT_DTYPE = np.dtype([("record", "<u4"), ("pos", "<u4"), ("pattern", "<u2"), ("mism", "u1"), ("flags", "u1")])
AMP_DTYPE = np.dtype([("hit_i", "<u4"), ("hit_j", "<u4"), ("record", "<u4"), ("start", "<u4"), ("end", "<u4"),
                      ("pair", "<u2"), ("orient", "u1"), ("flags", "u1"), ("tm", "<f8")])
assert HIT_DTYPE.itemsize == 12 and AMP_DTYPE.itemsize == 32


class AhError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ah_tm_params(ctypes.Structure):
    _fields_ = [("Na", ctypes.c_double), ("K", ctypes.c_double), ("Tris", ctypes.c_double), ("Mg", ctypes.c_double),
                ("dNTPs", ctypes.c_double), ("dnac1", ctypes.c_double), ("dnac2", ctypes.c_double),
                ("saltcorr", ctypes.c_int32), ("filter", ctypes.c_int32), ("min_tm", ctypes.c_double),
                ("variants", ctypes.c_int32), ("selfcomp", ctypes.c_int32), ("nn_table", ctypes.c_int32)]


class ah_plan_params(ctypes.Structure):
    _fields_ = [("min_len", ctypes.c_uint32), ("max_len", ctypes.c_uint32), ("orient_mask", ctypes.c_uint32),
                ("tm", ah_tm_params), ("extract", ctypes.c_int32), ("trim", ctypes.c_int32),
                ("fb_len", ctypes.c_uint32), ("rb_len", ctypes.c_uint32), ("autotune", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("hit_capacity", ctypes.c_uint64), ("amp_capacity", ctypes.c_uint64),
                ("arena_capacity", ctypes.c_uint64)]


class ah_plan_info(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("groups_per_thread", ctypes.c_int32), ("shift_mode", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("grid", ctypes.c_int32), ("slot_cap", ctypes.c_uint32),
                ("max_tile_sites", ctypes.c_uint32), ("hit_capacity", ctypes.c_uint64),
                ("amp_capacity", ctypes.c_uint64), ("arena_capacity", ctypes.c_uint64), ("n_hits", ctypes.c_uint64),
                ("n_amps", ctypes.c_uint64), ("n_kept", ctypes.c_uint64), ("arena_bytes", ctypes.c_uint64),
                ("autotune_ms", ctypes.c_double), ("best_scan_ms", ctypes.c_double), ("min_blocks", ctypes.c_int32),
                ("vote_windows", ctypes.c_int32), ("emit_queue", ctypes.c_int32)]


class ah_request(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_uint32), ("fwd", ctypes.c_void_p), ("rev", ctypes.c_void_p), ("k", ctypes.c_void_p),
                ("clamp", ctypes.c_uint8), ("first_record", ctypes.c_uint32), ("n_records", ctypes.c_uint32),
                ("min_len", ctypes.c_uint32), ("max_len", ctypes.c_uint32), ("orient_mask", ctypes.c_uint32),
                ("tm", ah_tm_params), ("extract", ctypes.c_int32), ("trim", ctypes.c_int32),
                ("fb_len", ctypes.c_uint32), ("rb_len", ctypes.c_uint32)]


class ah_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n_hits", ctypes.c_uint64), ("n_amps", ctypes.c_uint64),
                ("arena_bytes", ctypes.c_uint64), ("bases", ctypes.c_uint64), ("hits", ctypes.c_void_p),
                ("amps", ctypes.c_void_p), ("arena", ctypes.c_void_p), ("field_off", ctypes.c_void_p),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("error", ctypes.c_char * 256), ("t_stage", ctypes.c_double * 5)]


class ah_ctx_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("scan_launches", ctypes.c_uint64), ("scan_ms", ctypes.c_double),
                ("scan_bases", ctypes.c_uint64), ("jit_compiles", ctypes.c_uint64), ("jit_ms", ctypes.c_double),
                ("scan_ops_per_group", ctypes.c_int32), ("generic_scans", ctypes.c_uint64),
                ("generic_bases", ctypes.c_uint64), ("tm_generated", ctypes.c_uint64),
                ("tm_builtin", ctypes.c_uint64)]


class ah_batch_view(ctypes.Structure):
    _fields_ = [("n_records", ctypes.c_uint32), ("n_bases", ctypes.c_uint64), ("n_groups", ctypes.c_uint64),
                ("planes", ctypes.c_void_p), ("invalid", ctypes.c_void_p), ("rec_group", ctypes.c_void_p),
                ("rec_len", ctypes.c_void_p), ("genome_id", ctypes.c_void_p)]


# name -> (restype, argtypes)
_VP, _U32, _U64, _I32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_PVP = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = {
    "ah_ctx_create": (_I32, [_PVP, _I32, _VP]),
    "ah_ctx_destroy": (None, [_VP]),
    "ah_last_error": (ctypes.c_char_p, [_VP]),
    "ah_ctx_synchronize": (_I32, [_VP]),
    "ah_ctx_stream": (_VP, [_VP]),
    "ah_ctx_stats_get": (_I32, [_VP, ctypes.POINTER(ah_ctx_stats)]),
    "ah_ctx_stats_reset": (_I32, [_VP]),
    "ah_ctx_set_pairs_per_kernel": (_I32, [_VP, ctypes.c_int]),
    "ah_ctx_set_generic_scan": (_I32, [_VP, ctypes.c_int]),
    "ah_ctx_set_tm_kernel": (_I32, [_VP, ctypes.c_int]),
    "ah_ctx_set_tm_split": (_I32, [_VP, ctypes.c_uint64]),
    "ah_tm_kernel_check": (_I32, [_VP, _U32, ctypes.c_int, ctypes.c_char_p, ctypes.c_uint64]),
    "ah_ctx_set_timing": (_I32, [_VP, _I32]),
    "ah_ctx_set_scan_config": (_I32, [_VP, _I32, _I32, _I32, _I32]),
    "ah_ctx_set_scan_circuit": (_I32, [_VP, _I32, _I32, _I32]),
    "ah_pack_batch": (_I32, [_VP, _U32, _VP, _VP, _VP, _PVP]),
    "ah_pack_batch_device": (_I32, [_VP, _U32, _VP, _VP, _VP, _PVP]),
    "ah_fasta_pack": (_I32, [_VP, _VP, _U64, _VP, _PVP, _PVP]),
    "ah_fasta_pack_into": (_I32, [_VP, _VP, _U64, _VP, _PVP]),
    "ah_fasta_count": (_U32, [_VP]),
    "ah_fastq_pack": (_I32, [_VP, _VP, _U64, _VP, _PVP, _PVP, _PVP]),
    "ah_quals_count": (_U32, [_VP]),
    "ah_quals_copy": (_I32, [_VP, _VP, _U64, _VP]),
    "ah_quals_free": (None, [_VP]),
    "ah_extract_qualities": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "ah_amplicons_qual_copy": (_I32, [_VP, _VP, _U64]),
    "ah_amplicons_fastq": (_I32, [_U64, _VP, _VP, _VP, _VP, _U32, _VP, _VP, ctypes.c_int, _VP, _U64,
                                  ctypes.POINTER(ctypes.c_uint64)]),
    "ah_fasta_name": (ctypes.c_char_p, [_VP, _U32]),
    "ah_fasta_free": (None, [_VP]),
    "ah_fasta_names_copy": (_I32, [_VP, _VP, _U64, _VP]),
    "ah_amplicons_fasta": (_I32, [_U64, _VP, _VP, _VP, _U32, _VP, _VP, ctypes.c_int, _VP, _U64,
                                  ctypes.POINTER(ctypes.c_uint64)]),
    "ah_batch_export": (_I32, [_VP, _VP, ctypes.POINTER(ctypes.c_uint64), _VP, _VP]),
    "ah_batch_import": (_I32, [_VP, _VP, _VP, _U64, _VP, _VP]),
    "ah_batch_view_get": (_I32, [_VP, ctypes.POINTER(ah_batch_view)]),
    "ah_batch_slice": (_I32, [_VP, _VP, _U32, _U32, _PVP]),
    "ah_batch_create": (_I32, [_VP, _U32, _VP, _VP, _PVP]),
    "ah_batch_pack_range": (_I32, [_VP, _VP, _U32, _U32, _VP, _VP]),
    "ah_batch_free": (None, [_VP]),
    "ah_primers_create": (_I32, [_VP, _U32, _VP, _VP, _VP, ctypes.c_uint8, _PVP]),
    "ah_primers_free": (None, [_VP]),
    "ah_scan_primers": (_I32, [_VP, _VP, _VP, _PVP]),
    "ah_scan_primers_per_record": (_I32, [_VP, _VP, _VP, _PVP]),
    "ah_hits_count": (_I32, [_VP, ctypes.POINTER(ctypes.c_uint64)]),
    "ah_hits_device": (_I32, [_VP, _PVP, _PVP]),
    "ah_hits_copy": (_I32, [_VP, _VP, _U64]),
    "ah_hits_free": (None, [_VP]),
    "ah_pair_amplicons": (_I32, [_VP, _VP, _VP, _VP, _U32, _U32, _U32, _PVP]),
    "ah_pair_amplicons_noalloc": (_I32, [_VP, _VP, _U64, _VP, _VP, _U32, _U32, _U32, _VP, _U64,
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "ah_tm_filter": (_I32, [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(ah_tm_params)]),
    "ah_tm_duplexes": (_I32, [_VP, _U32, _VP, _VP, ctypes.POINTER(ah_tm_params), _VP]),
    "ah_tm_sites": (_I32, [_VP, _U32, _VP, _VP, _VP, _VP, ctypes.POINTER(ah_tm_params), _VP]),
    "ah_extract_barcodes": (_I32, [_VP, _VP, _VP, _VP, _VP, _I32, _U32, _U32]),
    "ah_amplicons_count": (_I32, [_VP, ctypes.POINTER(ctypes.c_uint64)]),
    "ah_amplicons_copy": (_I32, [_VP, _VP, _U64]),
    "ah_amplicons_arena_size": (_I32, [_VP, ctypes.POINTER(ctypes.c_uint64)]),
    "ah_amplicons_seq_copy": (_I32, [_VP, _VP, _U64, _VP, _U64]),
    "ah_amplicons_free": (None, [_VP]),
    "ah_plan_create": (_I32, [_VP, _VP, _VP, ctypes.POINTER(ah_plan_params), _PVP]),
    "ah_plan_launch": (_I32, [_VP]),
    "ah_plan_check": (_I32, [_VP]),
    "ah_plan_run": (_I32, [_VP]),
    "ah_plan_info_get": (_I32, [_VP, ctypes.POINTER(ah_plan_info)]),
    "ah_plan_copy_results": (_I32, [_VP, _VP, _U64, _VP, _U64, _VP, _U64, _VP, _U64]),
    "ah_plan_results": (_I32, [_VP, _PVP, _PVP]),
    "ah_plan_free": (None, [_VP]),
    "ah_server_create": (_I32, [_VP, _I32, _U64, _PVP]),
    "ah_server_submit": (_I32, [_VP, ctypes.POINTER(ah_request), ctypes.POINTER(ctypes.c_uint64)]),
    "ah_server_wait": (_I32, [_VP, _U64, ctypes.POINTER(ctypes.POINTER(ah_result))]),
    "ah_server_now": (_I32, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "ah_server_set_scan_mode": (_I32, [_VP, ctypes.c_int]),
    "ah_server_cancel": (_I32, [_VP, _U64]),
    "ah_server_request_bytes": (_I32, [_VP, ctypes.POINTER(ah_request), ctypes.POINTER(ctypes.c_uint64)]),
    "ah_server_memory": (_I32, [_VP, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                ctypes.POINTER(ctypes.c_uint64)]),
    "ah_server_inject_alloc_failures": (_I32, [_VP, ctypes.c_int]),
    "ah_ctx_inject_alloc_failures": (_I32, [_VP, ctypes.c_int]),
    "ah_plan_launch_host": (_I32, [_VP, _VP, _VP]),
    "ah_plan_launch_packed": (_I32, [_VP, _VP, ctypes.c_uint64, _VP, _VP]),
    "ah_plan_launch_fasta": (_I32, [_VP, _VP, ctypes.c_uint64]),
    "ah_fasta_pack_file": (_I32, [_VP, ctypes.c_char_p, _VP, _PVP, _PVP]),
    "ah_fastq_pack_file": (_I32, [_VP, ctypes.c_char_p, _VP, _PVP, _PVP, _PVP]),
    "ah_result_free": (None, [ctypes.POINTER(ah_result)]),
    "ah_server_destroy": (None, [_VP]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libah.so (built by ``paper_2511_00170_gb300.build``).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with `python -m paper_2511_00170_gb300.build` "
                              "(the engine has no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(st: int, ctx=None):
    if st != AH_OK:
        msg = load().ah_last_error(ctx).decode() if ctx else ""
        raise AhError(st, msg)


# ------------------------------------------------------------------------------------------ context
def ah_ctx_create(device: int = 0, stream: Optional[int] = None):
    out = ctypes.c_void_p()
    _check(load().ah_ctx_create(ctypes.byref(out), device, stream))
    return out


def ah_ctx_destroy(ctx) -> None:
    load().ah_ctx_destroy(ctx)


def ah_last_error(ctx) -> str:
    return load().ah_last_error(ctx).decode()


def ah_ctx_synchronize(ctx) -> None:
    _check(load().ah_ctx_synchronize(ctx), ctx)


def ah_ctx_stream(ctx) -> int:
    return load().ah_ctx_stream(ctx) or 0


def ah_ctx_stats_get(ctx) -> dict:
    s = ah_ctx_stats()
    _check(load().ah_ctx_stats_get(ctx, ctypes.byref(s)), ctx)
    return {f: getattr(s, f) for f, _ in ah_ctx_stats._fields_}


def ah_ctx_stats_reset(ctx) -> None:
    _check(load().ah_ctx_stats_reset(ctx), ctx)


def ah_ctx_set_pairs_per_kernel(ctx, pairs: int) -> None:
    _check(load().ah_ctx_set_pairs_per_kernel(ctx, int(pairs)), ctx)


def ah_ctx_set_generic_scan(ctx, mode: int) -> None:
    """0: generated scan kernels; 1: the generic (compile-free) kernel; 2: the generic kernel while the
    primer set's kernels compile; 3: generic on the first half of the tiles, generated on the rest."""
    _check(load().ah_ctx_set_generic_scan(ctx, int(mode)), ctx)


def ah_ctx_set_tm_kernel(ctx, mode: int) -> None:
    """Degenerate-site Tm kernel: 0 generated for the primer set; 1 built in; 2 built in while the
    generated one compiles."""
    _check(load().ah_ctx_set_tm_kernel(ctx, int(mode)), ctx)


def ah_ctx_set_tm_split(ctx, sites: int = 0) -> None:
    """Site capacity from which the generated Tm kernel runs as one launch per group of primers
    (0: the default, 2**64 - 1: never)."""
    _check(load().ah_ctx_set_tm_split(ctx, int(sites)), ctx)


def ah_tm_kernel_check(primers: Sequence[str], sm: int = 103) -> Tuple[int, str]:
    """Generate and compile (NVRTC, no device) the Tm kernel for these primers: (status, log)."""
    arr = (ctypes.c_char_p * len(primers))(*[p.encode() for p in primers])
    log = ctypes.create_string_buffer(1 << 16)
    st = load().ah_tm_kernel_check(ctypes.cast(arr, ctypes.c_void_p), len(primers), int(sm), log, len(log))
    return st, log.value.decode(errors="replace")


def ah_ctx_set_timing(ctx, enable: bool) -> None:
    _check(load().ah_ctx_set_timing(ctx, int(bool(enable))), ctx)


def ah_ctx_set_scan_config(ctx, threads: int = 256, groups_per_thread: int = 4, slot_cap: int = 256,
                           shift_mode: int = 0) -> None:
    _check(load().ah_ctx_set_scan_config(ctx, threads, groups_per_thread, slot_cap, shift_mode), ctx)


def ah_ctx_set_scan_circuit(ctx, min_blocks: int = 0, vote_windows: int = 1024, emit_queue: int = 0) -> None:
    """Register bound (blocks per SM, 0 none), the phase split's windows per vote and the candidate
    queue (1) or direct emission (0) of the generated scan kernel; a plan without autotuning uses
    them as set."""
    _check(load().ah_ctx_set_scan_circuit(ctx, min_blocks, vote_windows, emit_queue), ctx)


# ------------------------------------------------------------------------------------------ packing
def ah_pack_batch(ctx, seq: np.ndarray, offsets: np.ndarray, genome_ids: Optional[np.ndarray] = None):
    """Records are seq[offsets[r]:offsets[r+1]] of a contiguous host uint8 buffer (pinned is faster)."""
    seq = np.ascontiguousarray(seq).view(np.uint8).reshape(-1)
    offsets = np.asarray(offsets, dtype=np.uint64)
    n = len(offsets) - 1
    ptrs = (np.uint64(seq.ctypes.data) + offsets[:-1]).astype(np.uint64)
    lens = np.diff(offsets).astype(np.uint64)
    gid = None if genome_ids is None else np.ascontiguousarray(genome_ids, dtype=np.uint32)
    out = ctypes.c_void_p()
    _check(load().ah_pack_batch(ctx, n, ptrs.ctypes.data, lens.ctypes.data, None if gid is None else gid.ctypes.data,
                                ctypes.byref(out)), ctx)
    return out


def ah_pack_batch_device(ctx, d_seq: int, offsets: np.ndarray, genome_ids: Optional[np.ndarray] = None):
    """Records already in device memory at address d_seq; offsets (host) delimit them."""
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    gid = None if genome_ids is None else np.ascontiguousarray(genome_ids, dtype=np.uint32)
    out = ctypes.c_void_p()
    _check(load().ah_pack_batch_device(ctx, len(offsets) - 1, d_seq, offsets.ctypes.data,
                                       None if gid is None else gid.ctypes.data, ctypes.byref(out)), ctx)
    return out


def _names_of(h) -> List[str]:
    """The names held by an ah_fasta handle (bulk copy), then the handle freed."""
    L = load()
    try:
        n = L.ah_fasta_count(h)
        off = np.zeros(n + 1, dtype=np.uint64)
        _check(L.ah_fasta_names_copy(h, None, 0, off.ctypes.data))
        buf = ctypes.create_string_buffer(max(1, int(off[-1])))
        _check(L.ah_fasta_names_copy(h, buf, int(off[-1]), off.ctypes.data))
        raw = buf.raw[:int(off[-1])].decode("latin-1")
        return [raw[int(off[i]):int(off[i + 1])] for i in range(n)]
    finally:
        L.ah_fasta_free(h)


def ah_fasta_names_copy(names) -> Tuple[bytes, np.ndarray]:
    """(all names back to back, offsets) of an ah_fasta handle."""
    L = load()
    n = L.ah_fasta_count(names)
    off = np.zeros(n + 1, dtype=np.uint64)
    _check(L.ah_fasta_names_copy(names, None, 0, off.ctypes.data))
    buf = ctypes.create_string_buffer(max(1, int(off[-1])))
    _check(L.ah_fasta_names_copy(names, buf, int(off[-1]), off.ctypes.data))
    return buf.raw[:int(off[-1])], off


def ah_fasta_pack(ctx, text, genome_ids: Optional[np.ndarray] = None, n_bytes: Optional[int] = None):
    """FASTA text (bytes / numpy uint8 on the host, or a device address with n_bytes) parsed and packed
    on the device.  Returns (batch, names)."""
    keep = None
    if isinstance(text, int):
        addr, n = text, int(n_bytes)
    else:
        keep = np.frombuffer(text, dtype=np.uint8) if isinstance(text, (bytes, bytearray)) else \
            np.ascontiguousarray(text, dtype=np.uint8)
        addr, n = keep.ctypes.data, len(keep)
    gid = None if genome_ids is None else np.ascontiguousarray(genome_ids, dtype=np.uint32)
    out, names = ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().ah_fasta_pack(ctx, addr, n, None if gid is None else gid.ctypes.data, ctypes.byref(out),
                                ctypes.byref(names)), ctx)
    return out, _names_of(names)


def ah_fasta_pack_into(ctx, text, batch, n_bytes: Optional[int] = None, names: bool = False):
    """FASTA text packed into an existing batch of the same record lengths; returns the names if asked."""
    keep = None
    if isinstance(text, int):
        addr, n = text, int(n_bytes)
    else:
        keep = np.frombuffer(text, dtype=np.uint8) if isinstance(text, (bytes, bytearray)) else \
            np.ascontiguousarray(text, dtype=np.uint8)
        addr, n = keep.ctypes.data, len(keep)
    h = ctypes.c_void_p()
    _check(load().ah_fasta_pack_into(ctx, addr, n, batch, ctypes.byref(h) if names else None), ctx)
    return _names_of(h) if names else None


def ah_fastq_pack(ctx, text, genome_ids: Optional[np.ndarray] = None, n_bytes: Optional[int] = None,
                  names: bool = True):
    """FASTQ text (host bytes/array, or a device address with n_bytes) parsed on the device.  Returns
    (batch, quals, names or None); free quals with ah_quals_free."""
    keep = None
    if isinstance(text, int):
        addr, n = text, int(n_bytes)
    else:
        keep = np.frombuffer(text, dtype=np.uint8) if isinstance(text, (bytes, bytearray)) else \
            np.ascontiguousarray(text, dtype=np.uint8)
        addr, n = keep.ctypes.data, len(keep)
    gid = None if genome_ids is None else np.ascontiguousarray(genome_ids, dtype=np.uint32)
    out, q, h = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().ah_fastq_pack(ctx, addr, n, None if gid is None else gid.ctypes.data, ctypes.byref(out),
                                ctypes.byref(q), ctypes.byref(h) if names else None), ctx)
    return out, q, (_names_of(h) if names else None)


def ah_fasta_pack_file(ctx, path: str, genome_ids: Optional[np.ndarray] = None):
    """A FASTA file read, parsed and packed; returns (batch, names)."""
    gid = None if genome_ids is None else np.ascontiguousarray(genome_ids, dtype=np.uint32)
    out, names = ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().ah_fasta_pack_file(ctx, os.fsencode(path), None if gid is None else gid.ctypes.data,
                                     ctypes.byref(out), ctypes.byref(names)), ctx)
    return out, _names_of(names)


def ah_fastq_pack_file(ctx, path: str, genome_ids: Optional[np.ndarray] = None, names: bool = True):
    """A FASTQ file read, parsed and packed; returns (batch, quals, names or None)."""
    gid = None if genome_ids is None else np.ascontiguousarray(genome_ids, dtype=np.uint32)
    out, q, h = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().ah_fastq_pack_file(ctx, os.fsencode(path), None if gid is None else gid.ctypes.data,
                                     ctypes.byref(out), ctypes.byref(q), ctypes.byref(h) if names else None), ctx)
    return out, q, (_names_of(h) if names else None)


def ah_quals_count(quals) -> int:
    return int(load().ah_quals_count(quals))


def ah_quals_copy(quals) -> Tuple[bytes, np.ndarray]:
    """(all qualities back to back, record offsets)."""
    n = ah_quals_count(quals)
    off = np.zeros(n + 1, dtype=np.uint64)
    L = load()
    _check(L.ah_quals_copy(quals, None, 0, off.ctypes.data))
    total = int(off[-1])
    buf = ctypes.create_string_buffer(max(1, total))
    _check(L.ah_quals_copy(quals, buf, total, off.ctypes.data))
    return buf.raw[:total], off


def ah_quals_free(quals) -> None:
    load().ah_quals_free(quals)


def ah_extract_qualities(ctx, quals, batch, primers, hits, amps) -> None:
    _check(load().ah_extract_qualities(ctx, quals, batch, primers, hits, amps), ctx)


def ah_amplicons_qual_copy(amps, arena_bytes: int) -> bytes:
    buf = ctypes.create_string_buffer(max(1, arena_bytes))
    _check(load().ah_amplicons_qual_copy(amps, buf, arena_bytes))
    return buf.raw[:arena_bytes]


def ah_fasta_count(names) -> int:
    """Records of an ah_fasta handle (ah_fasta_pack's wrapper returns the names as a list)."""
    return int(load().ah_fasta_count(names))


def ah_fasta_name(names, i: int) -> Optional[str]:
    v = load().ah_fasta_name(names, int(i))
    return None if v is None else v.decode("latin-1")


def ah_fasta_free(names) -> None:
    load().ah_fasta_free(names)


def _cstrings(strings: Sequence[str]):
    """A C array of NUL-terminated strings for a string list: (objects to keep alive, its address).
    The strings go into one buffer and the pointer array is computed with numpy, which for millions
    of names is several times faster than a ctypes c_char_p array."""
    enc = [x.encode("latin-1") for x in strings]
    blob = np.frombuffer(b"\0".join(enc) + b"\0", dtype=np.uint8)
    lens = np.fromiter((len(e) + 1 for e in enc), dtype=np.uint64, count=len(enc))
    ptrs = np.empty(max(1, len(enc)), dtype=np.uint64)
    ptrs[0] = 0
    np.cumsum(lens[:-1], out=ptrs[1:len(enc)])
    ptrs += np.uint64(blob.ctypes.data)
    return (blob, ptrs), ptrs.ctypes.data


def _write_records(fn, args, out: Optional[np.ndarray]):
    """Run a two-call writer: the size, then the text into `out` (returning the bytes written) or
    into a new buffer (returning bytes)."""
    n = ctypes.c_uint64()
    _check(fn(*args, None, 0, ctypes.byref(n)))
    if out is not None:
        if out.dtype != np.uint8 or not out.flags.c_contiguous or not out.flags.writeable or out.size < n.value:
            raise ValueError(f"out must be a writable contiguous uint8 array of at least {n.value} bytes")
        _check(fn(*args, out.ctypes.data, n.value, ctypes.byref(n)))
        return n.value
    buf = np.empty(max(1, n.value), dtype=np.uint8)
    _check(fn(*args, buf.ctypes.data, n.value, ctypes.byref(n)))
    return buf[:n.value].tobytes()


def ah_amplicons_fasta(amps: np.ndarray, arena: bytes, field_off: np.ndarray, record_names: Sequence[str],
                       record_sources: Optional[Sequence[str]] = None, barcodes: bool = False,
                       out: Optional[np.ndarray] = None):
    """FASTA records with the headers of the paper's output (host formatting of copied results).
    Returns the text as bytes, or with `out` (a uint8 array) writes it there and returns its length."""
    amps = np.ascontiguousarray(amps, dtype=AMP_DTYPE)
    off = np.ascontiguousarray(field_off, dtype=np.uint64)
    arena = arena or b"\0"
    keep_n, names = _cstrings(record_names)
    keep_s, srcs = (None, None) if record_sources is None else _cstrings(record_sources)
    args = (len(amps), amps.ctypes.data, arena, off.ctypes.data, len(record_names), names, srcs, int(bool(barcodes)))
    return _write_records(load().ah_amplicons_fasta, args, out)


def ah_amplicons_fastq(amps: np.ndarray, arena: bytes, qual_arena: bytes, field_off: np.ndarray,
                       record_names: Sequence[str], record_sources: Optional[Sequence[str]] = None,
                       barcodes: bool = False, out: Optional[np.ndarray] = None):
    """FASTQ records: the FASTA headers with '@', the sequence, '+', the qualities.  Returns bytes, or
    with `out` writes there and returns the length."""
    amps = np.ascontiguousarray(amps, dtype=AMP_DTYPE)
    off = np.ascontiguousarray(field_off, dtype=np.uint64)
    arena, qual_arena = arena or b"\0", qual_arena or b"\0"
    keep_n, names = _cstrings(record_names)
    keep_s, srcs = (None, None) if record_sources is None else _cstrings(record_sources)
    args = (len(amps), amps.ctypes.data, arena, qual_arena, off.ctypes.data, len(record_names), names, srcs,
            int(bool(barcodes)))
    return _write_records(load().ah_amplicons_fastq, args, out)


def ah_batch_export(batch, planes: Optional[np.ndarray] = None, groups: Optional[np.ndarray] = None,
                    words: Optional[np.ndarray] = None):
    """Packed bases of a batch for storage: (planes uint32[n_groups, 2], invalid group indices uint64,
    invalid words uint32).  Caller arrays (e.g. page-locked) may be passed in; the lists are sized by
    a first counting call."""
    v = ah_batch_view_get(batch)
    if planes is None:
        planes = np.empty((v["n_groups"], 2), dtype=np.uint32)
    n = ctypes.c_uint64(0)
    _check(load().ah_batch_export(batch, None, ctypes.byref(n), None, None))
    if groups is None:
        groups = np.empty(n.value, dtype=np.uint64)
    if words is None:
        words = np.empty(n.value, dtype=np.uint32)
    n2 = ctypes.c_uint64(len(groups))
    _check(load().ah_batch_export(batch, planes.ctypes.data, ctypes.byref(n2), groups.ctypes.data, words.ctypes.data))
    return planes, groups[:n2.value], words[:n2.value]


def ah_batch_import(ctx, batch, planes: np.ndarray, groups: np.ndarray, words: np.ndarray) -> None:
    _check(load().ah_batch_import(ctx, batch, planes.ctypes.data, len(groups), groups.ctypes.data if len(groups) else None,
                                  words.ctypes.data if len(words) else None), ctx)


def ah_batch_view_get(batch) -> dict:
    v = ah_batch_view()
    _check(load().ah_batch_view_get(batch, ctypes.byref(v)))
    return {f: getattr(v, f) for f, _ in ah_batch_view._fields_}


def ah_batch_slice(ctx, db, first: int, count: int):
    out = ctypes.c_void_p()
    _check(load().ah_batch_slice(ctx, db, first, count, ctypes.byref(out)), ctx)
    return out


def ah_batch_create(ctx, lengths: np.ndarray, genome_ids: Optional[np.ndarray] = None):
    lens = np.ascontiguousarray(lengths, dtype=np.uint64)
    gid = None if genome_ids is None else np.ascontiguousarray(genome_ids, dtype=np.uint32)
    out = ctypes.c_void_p()
    _check(load().ah_batch_create(ctx, len(lens), lens.ctypes.data, None if gid is None else gid.ctypes.data,
                                  ctypes.byref(out)), ctx)
    return out


def ah_batch_pack_range(ctx, batch, first: int, d_seq: int, offsets: np.ndarray) -> None:
    """Pack records first .. first + len(offsets) - 2 from device memory (offsets start at 0)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    _check(load().ah_batch_pack_range(ctx, batch, first, len(offsets) - 1, d_seq, offsets.ctypes.data), ctx)


def ah_batch_free(batch) -> None:
    load().ah_batch_free(batch)


# ------------------------------------------------------------------------------------------ primers
def ah_primers_create(ctx, fwd: Sequence[str], rev: Sequence[str], k: Sequence[int], clamp: int):
    n = len(fwd)
    fa = (ctypes.c_char_p * n)(*[s.encode("ascii") for s in fwd])
    ra = (ctypes.c_char_p * n)(*[s.encode("ascii") for s in rev])
    ka = np.ascontiguousarray(np.asarray(k, dtype=np.uint8))
    out = ctypes.c_void_p()
    _check(load().ah_primers_create(ctx, n, ctypes.cast(fa, ctypes.c_void_p), ctypes.cast(ra, ctypes.c_void_p),
                                    ka.ctypes.data, clamp, ctypes.byref(out)), ctx)
    return out


def ah_primers_free(p) -> None:
    load().ah_primers_free(p)


# ------------------------------------------------------------------------------------------ scan
def ah_scan_primers(ctx, batch, primers):
    out = ctypes.c_void_p()
    _check(load().ah_scan_primers(ctx, batch, primers, ctypes.byref(out)), ctx)
    return out


def ah_scan_primers_per_record(ctx, batch, primers):
    out = ctypes.c_void_p()
    _check(load().ah_scan_primers_per_record(ctx, batch, primers, ctypes.byref(out)), ctx)
    return out


def ah_hits_count(hits) -> int:
    n = ctypes.c_uint64()
    _check(load().ah_hits_count(hits, ctypes.byref(n)))
    return n.value


def ah_hits_device(hits):
    d, off = ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().ah_hits_device(hits, ctypes.byref(d), ctypes.byref(off)))
    return d.value, off.value


def ah_hits_copy(hits) -> np.ndarray:
    n = ah_hits_count(hits)
    out = np.empty(n, dtype=HIT_DTYPE)
    _check(load().ah_hits_copy(hits, out.ctypes.data if n else None, n))
    return out


def ah_hits_free(hits) -> None:
    load().ah_hits_free(hits)


# ------------------------------------------------------------------------------------------ pairing
def ah_pair_amplicons(ctx, batch, primers, hits, min_len: int, max_len: int, orient_mask: int = 15):
    out = ctypes.c_void_p()
    _check(load().ah_pair_amplicons(ctx, batch, primers, hits, min_len, max_len, orient_mask, ctypes.byref(out)), ctx)
    return out


AH_PAIR_NOALLOC_MAX_SITES = 1 << 20


def ah_pair_amplicons_noalloc(stream: int, d_hits: int, n_hits: int, d_pair_offsets: int, d_pattern_len: int,
                              min_len: int, max_len: int, orient_mask: int, d_out: int, out_capacity: int) -> int:
    """Pairing on caller-owned device buffers, allocating nothing (see include/ah.h).  Returns the
    number of amplicons written to d_out."""
    n = ctypes.c_uint64()
    st = load().ah_pair_amplicons_noalloc(stream, d_hits, n_hits, d_pair_offsets, d_pattern_len, min_len, max_len,
                                          orient_mask, d_out, out_capacity, ctypes.byref(n))
    if st != AH_OK:
        raise AhError(st, f"ah_pair_amplicons_noalloc ({n.value} amplicons found)")
    return n.value


# ------------------------------------------------------------------------------------------ Tm
def tm_params(Na=50.0, K=0.0, Tris=0.0, Mg=0.0, dNTPs=0.0, dnac1=25.0, dnac2=25.0, saltcorr=5, min_tm=None,
              variants=0, selfcomp=0, filter=None, nn_table=0) -> ah_tm_params:
    """min_tm None: no threshold (flags bit0 then marks a defined Tm).  filter None: filter iff a
    threshold is given; False with a threshold only annotates the decision in the flags."""
    flt = (min_tm is not None) if filter is None else bool(filter)
    if flt and min_tm is None:
        raise ValueError("filtering needs min_tm")
    return ah_tm_params(Na, K, Tris, Mg, dNTPs, dnac1, dnac2, saltcorr, int(flt),
                        float("-inf") if min_tm is None else float(min_tm), int(variants), int(selfcomp),
                        int(nn_table))


def ah_tm_filter(ctx, batch, primers, hits, amps, params: ah_tm_params) -> None:
    _check(load().ah_tm_filter(ctx, batch, primers, hits, amps, ctypes.byref(params)), ctx)


def ah_tm_duplexes(ctx, seqs: Sequence[str], cseqs: Sequence[str], params: ah_tm_params) -> np.ndarray:
    n = len(seqs)
    sa = (ctypes.c_char_p * n)(*[s.encode("ascii") for s in seqs])
    ca = (ctypes.c_char_p * n)(*[s.encode("ascii") for s in cseqs])
    out = np.empty(n, dtype=np.float64)
    _check(load().ah_tm_duplexes(ctx, n, ctypes.cast(sa, ctypes.c_void_p), ctypes.cast(ca, ctypes.c_void_p),
                                 ctypes.byref(params), out.ctypes.data), ctx)
    return out


def ah_tm_sites(ctx, primers: Sequence[str], sites: Sequence[str], params: ah_tm_params,
                k: Optional[Sequence[int]] = None, clamp: Optional[Sequence[int]] = None) -> np.ndarray:
    """Per site: the maximum Tm over the primer's variants with at most k[i] mismatches and an exact
    clamp of clamp[i] bases (None: no limit / no clamp)."""
    n = len(primers)
    pa = (ctypes.c_char_p * n)(*[s.encode("ascii") for s in primers])
    sa = (ctypes.c_char_p * n)(*[s.encode("ascii") for s in sites])
    ka = None if k is None else np.ascontiguousarray(np.asarray(k, dtype=np.uint8))
    ca = None if clamp is None else np.ascontiguousarray(np.asarray(clamp, dtype=np.uint8))
    out = np.empty(n, dtype=np.float64)
    _check(load().ah_tm_sites(ctx, n, ctypes.cast(pa, ctypes.c_void_p), ctypes.cast(sa, ctypes.c_void_p),
                              None if ka is None else ka.ctypes.data, None if ca is None else ca.ctypes.data,
                              ctypes.byref(params), out.ctypes.data), ctx)
    return out


# ------------------------------------------------------------------------------------------ extraction
def ah_extract_barcodes(ctx, batch, primers, hits, amps, trim: bool, fb_len: int, rb_len: int) -> None:
    _check(load().ah_extract_barcodes(ctx, batch, primers, hits, amps, int(bool(trim)), fb_len, rb_len), ctx)


def ah_amplicons_count(amps) -> int:
    n = ctypes.c_uint64()
    _check(load().ah_amplicons_count(amps, ctypes.byref(n)))
    return n.value


def ah_amplicons_copy(amps) -> np.ndarray:
    n = ah_amplicons_count(amps)
    out = np.empty(n, dtype=AMP_DTYPE)
    _check(load().ah_amplicons_copy(amps, out.ctypes.data if n else None, n))
    return out


def ah_amplicons_arena_size(amps) -> int:
    n = ctypes.c_uint64()
    _check(load().ah_amplicons_arena_size(amps, ctypes.byref(n)))
    return n.value


def ah_amplicons_seq_copy(amps):
    """(arena bytes, offsets uint64[5n+1])"""
    n = ah_amplicons_count(amps)
    size = ctypes.c_uint64()
    _check(load().ah_amplicons_arena_size(amps, ctypes.byref(size)))
    arena = np.empty(max(1, size.value), dtype=np.uint8)
    off = np.empty(5 * n + 1, dtype=np.uint64)
    _check(load().ah_amplicons_seq_copy(amps, arena.ctypes.data, size.value, off.ctypes.data, len(off)))
    return arena[:size.value].tobytes(), off


def ah_amplicons_free(amps) -> None:
    load().ah_amplicons_free(amps)


# ------------------------------------------------------------------------------------------ plans
def plan_params(min_len, max_len, orient_mask=15, tm: Optional[ah_tm_params] = None, extract=True, trim=False, fb_len=0,
                rb_len=0, autotune=False, persistent=-1, hit_capacity=0, amp_capacity=0, arena_capacity=0) -> ah_plan_params:
    return ah_plan_params(min_len, max_len, orient_mask, tm if tm is not None else tm_params(), int(bool(extract)),
                          int(bool(trim)), fb_len, rb_len, int(bool(autotune)), persistent, hit_capacity, amp_capacity,
                          arena_capacity)


def ah_plan_create(ctx, batch, primers, params: ah_plan_params):
    out = ctypes.c_void_p()
    _check(load().ah_plan_create(ctx, batch, primers, ctypes.byref(params), ctypes.byref(out)), ctx)
    return out


def ah_plan_launch(plan, ctx=None) -> None:
    _check(load().ah_plan_launch(plan), ctx)


def ah_plan_check(plan, ctx=None) -> None:
    _check(load().ah_plan_check(plan), ctx)


def ah_plan_run(plan, ctx=None) -> None:
    _check(load().ah_plan_run(plan), ctx)


def ah_plan_info_get(plan) -> dict:
    i = ah_plan_info()
    _check(load().ah_plan_info_get(plan, ctypes.byref(i)))
    return {f: getattr(i, f) for f, _ in ah_plan_info._fields_}


def ah_plan_copy_results(plan, ctx, hits: Optional[np.ndarray], amps: Optional[np.ndarray],
                         arena: Optional[np.ndarray], field_off: Optional[np.ndarray]) -> None:
    """Copy the last run's results into caller arrays (HIT_DTYPE, AMP_DTYPE, uint8, uint64; any may be
    None); the counts are in ah_plan_info_get afterwards."""
    def buf(a):
        return (None, 0) if a is None else (a.ctypes.data, len(a))
    h, a, r, f = buf(hits), buf(amps), buf(arena), buf(field_off)
    _check(load().ah_plan_copy_results(plan, h[0], h[1], a[0], a[1], r[0], r[1], f[0], f[1]), ctx)


def ah_plan_results(plan, ctx=None):
    h, a = ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().ah_plan_results(plan, ctypes.byref(h), ctypes.byref(a)), ctx)
    return h, a


def ah_plan_free(plan) -> None:
    load().ah_plan_free(plan)


# ------------------------------------------------------------------------------------------ serving
def ah_server_create(db, n_slots: int = 4, memory_budget: int = 0):
    out = ctypes.c_void_p()
    _check(load().ah_server_create(db, n_slots, memory_budget, ctypes.byref(out)))
    return out


def _request(fwd, rev, k, clamp, first_record, n_records, min_len, max_len, orient_mask=15, tm=None, extract=True,
             trim=False, fb_len=0, rb_len=0):
    """An ah_request and the buffers it points to (kept alive with it)."""
    n = len(fwd)
    fa = (ctypes.c_char_p * n)(*[x.encode("ascii") for x in fwd])
    ra = (ctypes.c_char_p * n)(*[x.encode("ascii") for x in rev])
    ka = np.ascontiguousarray(np.asarray(k, dtype=np.uint8))
    r = ah_request(n, ctypes.cast(fa, ctypes.c_void_p), ctypes.cast(ra, ctypes.c_void_p), ka.ctypes.data, clamp,
                   first_record, n_records, min_len, max_len, orient_mask, tm if tm is not None else tm_params(),
                   int(bool(extract)), int(bool(trim)), fb_len, rb_len)
    return r, (fa, ra, ka)


def ah_server_submit(server, fwd: Sequence[str], rev: Sequence[str], k: Sequence[int], clamp: int, first_record: int,
                     n_records: int, min_len: int, max_len: int, orient_mask: int = 15,
                     tm: Optional[ah_tm_params] = None, extract: bool = True, trim: bool = False, fb_len: int = 0,
                     rb_len: int = 0) -> int:
    r, keep = _request(fwd, rev, k, clamp, first_record, n_records, min_len, max_len, orient_mask, tm, extract, trim,
                       fb_len, rb_len)
    t = ctypes.c_uint64()
    _check(load().ah_server_submit(server, ctypes.byref(r), ctypes.byref(t)))
    return t.value


def ah_server_request_bytes(server, **req) -> int:
    """Device bytes the server reserves when it admits this request (same keywords as ah_server_submit)."""
    r, keep = _request(**req)
    b = ctypes.c_uint64()
    _check(load().ah_server_request_bytes(server, ctypes.byref(r), ctypes.byref(b)))
    return b.value


def ah_server_cancel(server, ticket: int) -> None:
    _check(load().ah_server_cancel(server, ticket))


def ah_server_memory(server) -> dict:
    b, r, p = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().ah_server_memory(server, ctypes.byref(b), ctypes.byref(r), ctypes.byref(p)))
    return {"budget": b.value, "reserved": r.value, "reserved_peak": p.value}


def ah_server_inject_alloc_failures(server, n: int) -> None:
    _check(load().ah_server_inject_alloc_failures(server, int(n)))


def ah_plan_launch_packed(plan, planes: np.ndarray, inv_groups: np.ndarray, inv_words: np.ndarray, ctx=None) -> None:
    """The plan's step on 2-bit batches in host memory (planes, sparse invalid words as ah_batch_export
    writes them), the scan overlapping the upload."""
    g = np.ascontiguousarray(inv_groups, dtype=np.uint64)
    w = np.ascontiguousarray(inv_words, dtype=np.uint32)
    _check(load().ah_plan_launch_packed(plan, planes.ctypes.data, len(g), g.ctypes.data if len(g) else None,
                                        w.ctypes.data if len(w) else None), ctx)


def ah_plan_launch_fasta(plan, text_ptr: int, n_bytes: int, ctx=None) -> None:
    """The plan's step on FASTA text at address text_ptr (host or device), records matching the
    plan's batch; the parse, the packing and the scan overlap the upload."""
    _check(load().ah_plan_launch_fasta(plan, text_ptr, int(n_bytes)), ctx)


def ah_plan_launch_host(plan, h_seq: int, offsets: np.ndarray, ctx=None) -> None:
    """The plan's step on genomes in host memory at address h_seq (records at offsets, uint64,
    n_records + 1 entries), the scan overlapping the upload."""
    offs = np.ascontiguousarray(offsets, dtype=np.uint64)
    _check(load().ah_plan_launch_host(plan, h_seq, offs.ctypes.data), ctx)


def ah_ctx_inject_alloc_failures(ctx, n: int) -> None:
    _check(load().ah_ctx_inject_alloc_failures(ctx, int(n)), ctx)


def ah_server_wait(server, ticket: int) -> dict:
    """Result of one request as host numpy arrays and timings (the C result is freed here)."""
    p = ctypes.POINTER(ah_result)()
    st = load().ah_server_wait(server, ticket, ctypes.byref(p))
    if not p:
        raise AhError(st, "ah_server_wait: unknown ticket")
    r = p.contents
    try:
        if st != AH_OK:
            raise AhError(st, r.error.decode(errors="replace"))
        hits = np.ctypeslib.as_array(ctypes.cast(r.hits, ctypes.POINTER(ctypes.c_uint8)), (r.n_hits * 12,)).copy() \
            .view(HIT_DTYPE) if r.n_hits else np.empty(0, HIT_DTYPE)
        amps = np.ctypeslib.as_array(ctypes.cast(r.amps, ctypes.POINTER(ctypes.c_uint8)), (r.n_amps * 32,)).copy() \
            .view(AMP_DTYPE) if r.n_amps else np.empty(0, AMP_DTYPE)
        arena = ctypes.string_at(r.arena, r.arena_bytes) if r.arena else None
        off = np.ctypeslib.as_array(ctypes.cast(r.field_off, ctypes.POINTER(ctypes.c_uint64)),
                                    (5 * r.n_amps + 1,)).copy() if r.field_off else None
        return {"hits": hits, "amps": amps, "arena": arena, "field_off": off, "bases": r.bases,
                "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done, "t_stage": list(r.t_stage)}
    finally:
        load().ah_result_free(p)


def ah_server_set_scan_mode(server, mode: int) -> None:
    """Generic-scan mode of requests admitted from now on (0 generated, 1 generic, 2 generic while compiling)."""
    _check(load().ah_server_set_scan_mode(server, int(mode)))


def ah_server_now(server) -> float:
    t = ctypes.c_double()
    _check(load().ah_server_now(server, ctypes.byref(t)))
    return t.value


def ah_server_destroy(server) -> None:
    load().ah_server_destroy(server)


def ah_result_free(result) -> None:
    """Free a raw ah_result pointer (ah_server_wait already frees the ones it converts)."""
    load().ah_result_free(result)
