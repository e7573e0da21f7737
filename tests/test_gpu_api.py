"""Error behaviour of the C ABI as include/ah.h documents it (needs a GPU): invalid arguments are
refused with AH_EINVAL and a message, nothing is half-made, and the context stays usable."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2511_00170_gb300 import ah

    ctx = ah.ah_ctx_create(0)
    wl = synth.random_small(3, n_records=4, len_lo=200, len_hi=600, n_pairs=1, plant=2)
    batch = ah.ah_pack_batch(ctx, wl.seq, wl.offsets)
    yield ah, ctx, wl, batch
    ah.ah_batch_free(batch)
    ah.ah_ctx_destroy(ctx)


def _refused(ah, ctx, status, fn, *a, **kw):
    with pytest.raises(ah.AhError) as e:
        fn(*a, **kw)
    assert e.value.status == status, (e.value.status, str(e.value))
    assert ah.ah_last_error(ctx)


def _still_works(ah, ctx, wl, batch):
    pr = ah.ah_primers_create(ctx, wl.fwd, wl.rev, wl.k, wl.clamp)
    try:
        h = ah.ah_scan_primers(ctx, batch, pr)
        ah.ah_hits_free(h)
    finally:
        ah.ah_primers_free(pr)
    ah.ah_ctx_synchronize(ctx)


@pytest.mark.parametrize("fwd,rev,k,clamp", [
    (["ACGTXACGT"], ["ACGTACGT"], [1], 2),        # not an IUPAC code
    (["A" * 33], ["ACGTACGT"], [1], 2),           # longer than 32
    (["ACGTACGT"], ["ACGTACGT"], [16], 2),        # k above 15
    (["ACGTACGT"], ["ACGTACGT"], [9], 2),         # k above the primer length
    (["ACGTACGT"], ["ACGTAC"], [1], 7),           # clamp longer than a primer
    ([], [], [], 2),                              # no pairs
])
def test_primers_refused(env, fwd, rev, k, clamp):
    ah, ctx, wl, batch = env
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_primers_create, ctx, fwd, rev, k, clamp)
    _still_works(ah, ctx, wl, batch)


def test_tm_parameters_refused(env):
    ah, ctx, wl, batch = env
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_tm_duplexes, ctx, ["ACGT"], ["TGCA"], ah.tm_params(saltcorr=8))
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_tm_duplexes, ctx, ["ACGT"], ["TGCA"], ah.tm_params(Na=0, saltcorr=7))
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_tm_duplexes, ctx, ["ACGT"], ["TGCA"], ah.tm_params(selfcomp=2))
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_tm_duplexes, ctx, ["ACGT"], ["TGCA"], ah.tm_params(dnac1=1, dnac2=4))
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_tm_duplexes, ctx, ["ACGT"], ["TGCA"], ah.tm_params(variants=2))
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_tm_duplexes, ctx, ["ACGT"], ["TGC"], ah.tm_params())   # lengths differ
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_tm_duplexes, ctx, ["ACGN"], ["TGCA"], ah.tm_params())  # not a base
    # ah_tm_sites: a mismatch budget above 15 and below the length, a clamp longer than the primer
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_tm_sites, ctx, ["ACGTACGTACGTACGTACGT"], ["ACGTACGTACGTACGTACGT"],
             ah.tm_params(), k=[16])
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_tm_sites, ctx, ["ACGTA"], ["ACGTA"], ah.tm_params(), k=[1], clamp=[6])
    _still_works(ah, ctx, wl, batch)


def test_batch_ranges_refused(env):
    import torch

    ah, ctx, wl, batch = env
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_batch_slice, ctx, batch, wl.n_records - 1, 2)
    lens = wl.lengths().astype(np.uint64)
    b = ah.ah_batch_create(ctx, lens)
    try:
        d = torch.from_numpy(wl.seq).cuda()
        offs = wl.offsets.astype(np.uint64)
        _refused(ah, ctx, ah.AH_EINVAL, ah.ah_batch_pack_range, ctx, b, 1, d.data_ptr(), offs)      # past the end
        bad = offs.copy()
        bad[1] += 1
        _refused(ah, ctx, ah.AH_EINVAL, ah.ah_batch_pack_range, ctx, b, 0, d.data_ptr(), bad)       # length differs
    finally:
        ah.ah_batch_free(b)
    _still_works(ah, ctx, wl, batch)


def test_context_settings_refused(env):
    ah, ctx, wl, batch = env
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_ctx_set_scan_config, ctx, 100, 4, 256, 0)   # not a multiple of 32
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_ctx_set_scan_config, ctx, 256, 4, 300, 0)   # slots not a power of 2
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_ctx_set_scan_config, ctx, 256, 4, 256, 3)   # no such shift mode
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_ctx_set_scan_circuit, ctx, 33, 1024)        # bound too high
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_ctx_set_scan_circuit, ctx, 0, 0)            # no windows
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_ctx_set_scan_circuit, ctx, 0, (1 << 20) + 1)
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_ctx_set_scan_circuit, ctx, 0, 1024, 2)       # no such emission
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_ctx_set_pairs_per_kernel, ctx, 257)
    _refused(ah, ctx, ah.AH_EINVAL, ah.ah_ctx_set_generic_scan, ctx, 4)
    _still_works(ah, ctx, wl, batch)


def test_plan_window_refused(env):
    ah, ctx, wl, batch = env
    pr = ah.ah_primers_create(ctx, wl.fwd, wl.rev, wl.k, wl.clamp)
    try:
        _refused(ah, ctx, ah.AH_EINVAL, ah.ah_plan_create, ctx, batch, pr, ah.plan_params(500, 100))
    finally:
        ah.ah_primers_free(pr)
    _still_works(ah, ctx, wl, batch)


def test_server_requests_refused(env):
    ah, ctx, wl, batch = env
    srv = ah.ah_server_create(batch, n_slots=1)
    try:
        with pytest.raises(ah.AhError) as e:
            ah.ah_server_submit(srv, wl.fwd, wl.rev, wl.k, wl.clamp, wl.n_records - 1, 2, 10, 500)   # past the end
        assert e.value.status == ah.AH_EINVAL
        with pytest.raises(ah.AhError) as e:
            ah.ah_server_submit(srv, [], [], [], wl.clamp, 0, 1, 10, 500)                     # no pairs
        assert e.value.status == ah.AH_EINVAL
        # a request whose primers are invalid is admitted and fails alone, with its message
        t = ah.ah_server_submit(srv, ["ACGTXACGT"], wl.rev, wl.k, wl.clamp, 0, 1, 10, 500)
        with pytest.raises(ah.AhError) as e:
            ah.ah_server_wait(srv, t)
        assert e.value.status == ah.AH_EINVAL
        ok = ah.ah_server_wait(srv, ah.ah_server_submit(srv, wl.fwd, wl.rev, wl.k, wl.clamp, 0, wl.n_records, 10, 500))
        assert len(ok["hits"]) >= 0
        with pytest.raises(ah.AhError) as e:
            ah.ah_server_set_scan_mode(srv, 3)
        assert e.value.status == ah.AH_EINVAL
    finally:
        ah.ah_server_destroy(srv)
