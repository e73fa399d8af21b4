"""C-ABI argument checks that return before any device work, so they run on
a machine without a GPU: null handles and buffers, empty batches, option
ranges, and the size limits of the no-allocation residual.  Buffers passed
where a check must fail first are fake addresses that are never read."""

import ctypes as C

import pytest

FAKE = 256  # a non-null address the library must not dereference in these calls


@pytest.fixture(scope="module")
def hz():
    import paper_2606_21695_gb300 as pkg

    return pkg


def _status(exc_info):
    return exc_info.value.status


def test_null_handles_are_invalid_arguments(hz):
    lib = hz.load()
    assert lib.hz_mesh_num_nodes(None, None) == hz.HZ_ERR_INVALID_ARG
    assert lib.hz_mesh_node_coords(None, None) == hz.HZ_ERR_INVALID_ARG
    n = C.c_int64()
    assert lib.hz_lambda_size(None, C.byref(n)) == hz.HZ_ERR_INVALID_ARG
    with pytest.raises(hz.HzError) as e:
        hz.hz_sweep(None, hz.HZ_FP64, 10, 1, 0.0, FAKE, FAKE + 64)
    assert _status(e) == hz.HZ_ERR_INVALID_ARG
    with pytest.raises(hz.HzError) as e:
        hz.hz_sweep_rect(None, hz.HZ_FP64, 10, 1, 0.0, (0, 0, 1, 1), FAKE, FAKE + 64)
    assert _status(e) == hz.HZ_ERR_INVALID_ARG
    with pytest.raises(hz.HzError) as e:
        hz.hz_lambda_gather(None, FAKE, 1, FAKE, FAKE)
    assert _status(e) == hz.HZ_ERR_INVALID_ARG
    with pytest.raises(hz.HzError) as e:
        hz.hz_server_stats(None)
    assert _status(e) == hz.HZ_ERR_INVALID_ARG
    hz.hz_server_destroy(None)  # a no-op
    hz.hz_mesh_destroy(None)
    hz.hz_problem_destroy(None)


def test_error_message_names_the_failure(hz):
    with pytest.raises(hz.HzError):
        hz.hz_mesh_create(0, 1, 0, 1, 10, 10, 2, 3, 5)
    assert hz.hz_last_error()  # a message for the calling thread
    lib = hz.load()
    assert lib.hz_last_error(None, 16) == hz.HZ_ERR_INVALID_ARG


def test_sweep_rejects_aliased_transmission_buffers(hz):
    """The alias check reads no field of the problem (a fake handle)."""
    with pytest.raises(hz.HzError) as e:
        hz.hz_sweep(C.c_void_p(FAKE), hz.HZ_FP64, 10, 1, 0.0, FAKE, FAKE)
    assert _status(e) == hz.HZ_ERR_INVALID_ARG and "alias" in str(e.value)


def test_empty_and_malformed_batches(hz):
    st, sts, us, reps = hz.hz_solve_batch([], [])
    assert st == hz.HZ_OK and sts == [] and us == [] and reps == []
    with pytest.raises(hz.HzError) as e:
        hz.hz_solve_batch([None], [5], want_u=False)
    assert _status(e) == hz.HZ_ERR_INVALID_ARG
    lib = hz.load()
    sts = (C.c_int32 * 1)()
    assert lib.hz_solve_batch(None, 1, None, 0, None, None, sts) == hz.HZ_ERR_INVALID_ARG
    assert lib.hz_solve_batch((C.c_void_p * 1)(), -1, None, 0, None, None, sts) == hz.HZ_ERR_INVALID_ARG


def test_lambda_slot_calls_check_counts(hz):
    lib = hz.load()
    # negative counts and null buffers with a positive count are refused;
    # a zero count with no buffers is a no-op, before the problem is used
    fake_pr = C.c_void_p(FAKE)
    assert lib.hz_lambda_gather(fake_pr, None, -1, None, None, None) == hz.HZ_ERR_INVALID_ARG
    assert lib.hz_lambda_scatter(fake_pr, None, 3, None, None, None) == hz.HZ_ERR_INVALID_ARG
    assert lib.hz_lambda_gather(fake_pr, None, 0, None, None, None) == hz.HZ_OK
    assert lib.hz_lambda_scatter(fake_pr, None, 0, None, None, None) == hz.HZ_OK


def test_peak_measurement_arguments(hz):
    with pytest.raises(hz.HzError) as e:
        hz.hz_fma_peak(hz.HZ_FP64, 0)
    assert _status(e) == hz.HZ_ERR_INVALID_ARG
    with pytest.raises(hz.HzError) as e:
        hz.hz_fma_peak(hz.HZ_BF16_TRIAL, 10)
    assert _status(e) == hz.HZ_ERR_INVALID_ARG


def test_noalloc_residual_limits_are_checked_on_the_host(hz):
    m = hz.hz_mesh_create(0, 1, 0, 1, 8192, 8192, 7, 8192, 8192)  # 57345^2 nodes, host-side only
    try:
        with pytest.raises(hz.HzError) as e:
            hz.hz_residual_noalloc(m, 1.0, FAKE, FAKE, FAKE, FAKE, FAKE)
        assert _status(e) == hz.HZ_ERR_UNSUPPORTED and "too large" in str(e.value)
        with pytest.raises(hz.HzError) as e:
            hz.hz_residual_noalloc(m, 0.0, FAKE, FAKE, FAKE, FAKE, FAKE)
        assert _status(e) == hz.HZ_ERR_INVALID_ARG
        with pytest.raises(hz.HzError) as e:
            hz.hz_residual_noalloc(m, 1.0, None, FAKE, FAKE, FAKE, FAKE)
        assert _status(e) == hz.HZ_ERR_INVALID_ARG
    finally:
        hz.hz_mesh_destroy(m)
    m = hz.hz_mesh_create(0, 1, 0, 100, 4, 600000, 1, 4, 600000)  # 5 x 600001 nodes: 75001 block rows
    try:
        with pytest.raises(hz.HzError) as e:
            hz.hz_residual_noalloc(m, 1.0, FAKE, FAKE, FAKE, FAKE, FAKE)
        assert _status(e) == hz.HZ_ERR_UNSUPPORTED and "node rows" in str(e.value)
    finally:
        hz.hz_mesh_destroy(m)


def test_options_struct_layout_matches_the_library(hz):
    """hz_default_opts (host only) fills the binding's struct with the
    documented defaults, last field included, and writes nothing past it."""
    class Guarded(C.Structure):
        _fields_ = [("opts", hz.hz_solve_opts), ("guard", C.c_uint8 * 64)]

    g = Guarded()
    C.memset(C.addressof(g.guard), 0xA5, 64)
    hz.load().hz_default_opts(C.byref(g.opts))
    assert bytes(g.guard) == b"\xa5" * 64
    o = g.opts
    assert (o.precision, o.tol, o.max_sweeps, o.outer, o.gmres_restart, o.wh_iters) == \
           (hz.HZ_FP64, 1e-8, 2000, hz.HZ_OUTER_GMRES, 60, 20)
    assert (o.wh_tol, o.nt_override, o.cfl, o.inner_tol, o.max_refine) == (0.0, 0, 0.9, 1e-2, 20)
    assert (o.autotune, o.wh_adaptive, o.pack, o.graphs, o.gs_passes, o.wh_warm) == (1, 0, 1, 1, 1, 0)
    assert (o.refine, o.refine_restart) == (hz.HZ_REFINE_DEFECT, 30)
    # the binding's keyword form sets fields by name over the same defaults
    k = hz.hz_default_opts(refine=hz.HZ_REFINE_FGMRES, refine_restart=60, tol=1e-9)
    assert (k.refine, k.refine_restart, k.tol, k.gmres_restart) == (hz.HZ_REFINE_FGMRES, 60, 1e-9, 60)
