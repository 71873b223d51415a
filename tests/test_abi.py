"""The C ABI without a GPU: the library loads, exports every entry point that
include/ptsdf.h declares, the Python binding names the same calls, and the
host-side argument checks reject bad input before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ptsdf.h")


@pytest.fixture(scope="module")
def abi():
    from paper_2607_16946_b300 import build
    build.build()
    from paper_2607_16946_b300 import _abi
    return _abi


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"PTSDF_API\s+[\w\s\*]+?\b(sdf_\w+)\s*\(", txt)))


def test_header_declares_calls():
    names = declared_functions()
    for required in ("sdf_build", "sdf_query", "sdf_query_host", "sdf_destroy", "sdf_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(abi):
    L = ctypes.CDLL(abi.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), name


def test_binding_covers_header(abi):
    assert set(declared_functions()) == set(abi.SIGNATURES)


def test_host_side_validation(abi):
    L = abi.lib()
    o = abi.sdf_query_opts()
    assert L.sdf_opts_default(ctypes.byref(o)) == abi.SDF_OK
    assert o.C == 64.0 and o.lambda_mode == abi.SDF_LAMBDA_GLOBAL and o.split_n == 0
    assert L.sdf_opts_default(None) == abi.SDF_EINVAL
    h = ctypes.c_void_p()
    assert L.sdf_build(None, None, None, 0, None, ctypes.byref(h)) == abi.SDF_EINVAL
    assert b"n must be" in L.sdf_last_error()
    assert L.sdf_build(None, None, None, 10, None, ctypes.byref(h)) == abi.SDF_EINVAL
    assert L.sdf_build(None, None, None, 10, None, None) == abi.SDF_EINVAL
    assert L.sdf_query(None, None, 0, None, None, None) == abi.SDF_EINVAL
    assert L.sdf_query_host(None, None, 5, None, None, None) == abi.SDF_EINVAL
    assert L.sdf_destroy(None) == abi.SDF_OK
    code = ctypes.c_int32()
    assert L.sdf_device_status(None, None, ctypes.byref(code)) == abi.SDF_EINVAL
    assert L.sdf_version().startswith(b"ptsdf")


def test_missing_library_fails_loudly(abi, monkeypatch, tmp_path):
    monkeypatch.setattr(abi, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(abi, "_lib", None)
    with pytest.raises(FileNotFoundError):
        abi.lib()


def test_serve_host_side_validation(abi):
    from paper_2607_16946_b300 import serve
    L = abi.lib()
    h = ctypes.c_void_p()
    assert L.sdf_serve_create(None, ctypes.byref(h)) == abi.SDF_EINVAL
    bad = serve.sdf_serve_config(1 << 20, 0, 1, 0, 0, 0, 0)
    assert L.sdf_serve_create(ctypes.byref(bad), ctypes.byref(h)) == abi.SDF_EINVAL
    bad = serve.sdf_serve_config(0, 1, 1, 0, 0, 0, 0)
    assert L.sdf_serve_create(ctypes.byref(bad), ctypes.byref(h)) == abi.SDF_EINVAL
    bad = serve.sdf_serve_config(1 << 20, 1, 1, 0, 7, 0, 0)
    assert L.sdf_serve_create(ctypes.byref(bad), ctypes.byref(h)) == abi.SDF_EINVAL
    # express streams: a negative or NaN threshold, or one stream for two classes
    for express, streams in ((-1.0, 4), (float("nan"), 4), (1.0, 1)):
        bad = serve.sdf_serve_config(1 << 20, 1, streams, 0, 0, 0, 0, express)
        assert L.sdf_serve_create(ctypes.byref(bad), ctypes.byref(h)) == abi.SDF_EINVAL
        assert b"express_gpairs" in L.sdf_last_error()
    assert L.sdf_serve_submit(None, None, None) == abi.SDF_EINVAL
    assert L.sdf_serve_poll(None, 1, 0, None) == abi.SDF_EINVAL
    assert L.sdf_serve_shutdown(None) == abi.SDF_OK
    # the ctypes structures match the C layout (sizes from include/ptsdf.h)
    assert ctypes.sizeof(serve.sdf_serve_config) == 40
    assert ctypes.sizeof(serve.sdf_request_stats) == 48
    assert ctypes.sizeof(serve.sdf_request) == 16 + 5 * 8 + ctypes.sizeof(abi.sdf_query_opts)


def _refusals(abi):
    """(call, expected message) for a refusal of every entry point taking a
    cloud or device buffers, each decided before any CUDA call."""
    L = abi.lib()
    o = abi.make_opts()
    f, i64, i32, d = ctypes.c_float(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
    fake = ctypes.c_void_p(16)          # a non-NULL device address the checks must refuse before using
    one = (ctypes.c_float * 3)(1.0, 1.0, 1.0)
    return [
        (lambda: L.sdf_query_grad(None, None, 4, None, None, None, ctypes.byref(o), None), b"sdf_query_grad: cloud"),
        (lambda: L.sdf_query_laplacian(None, None, 4, None, None, None, ctypes.byref(o), None),
         b"sdf_query_laplacian: cloud"),
        (lambda: L.sdf_project_level_set(None, None, 4, 0.0, 3, 0.0, None, None, None, ctypes.byref(o), None),
         b"sdf_project_level_set: cloud"),
        (lambda: L.sdf_backward_params(None, None, 4, None, None, None, ctypes.byref(o), None),
         b"sdf_backward_params: cloud"),
        (lambda: L.sdf_trace(None, None, None, 4, 48, 1e-4, 6.0, None, None, None, ctypes.byref(o), None),
         b"sdf_trace: cloud"),
        (lambda: L.sdf_query_noalloc(None, None, 4, None, ctypes.byref(o), None), b"sdf_query_noalloc: cloud"),
        # the allocation-free query refuses what sdf_query refuses, before looking at the cloud
        (lambda: L.sdf_query_noalloc(None, None, 4, None, ctypes.byref(abi.make_opts(formula=7)), None),
         b"sdf_query_noalloc: unknown formula"),
        (lambda: L.sdf_query_noalloc(None, None, 4, None, ctypes.byref(abi.make_opts(
            formula=abi.SDF_FORMULA_LSE, lambda_mode=abi.SDF_LAMBDA_FIXED, fixed_lambda=0.0)), None),
         b"sdf_query_noalloc: the log-sum-exp distance needs fixed_lambda > 0"),
        (lambda: L.sdf_query_noalloc(None, None, 4, None, ctypes.byref(abi.make_opts(C=-1.0)), None),
         b"sdf_query_noalloc: C must be > 0"),
        # and what it leaves out
        (lambda: L.sdf_query_noalloc(None, None, 4, None, ctypes.byref(abi.make_opts(
            lambda_mode=abi.SDF_LAMBDA_RADIUS, fixed_lambda=10.0)), None), b"GLOBAL or FIXED lambda only"),
        (lambda: L.sdf_query_noalloc(None, None, 4, None, ctypes.byref(abi.make_opts(precision=abi.SDF_F16X2)),
                                     None), b"sdf_query_noalloc: FP32 only"),
        (lambda: L.sdf_query_noalloc(None, None, 4, None, ctypes.byref(abi.make_opts(engine=abi.SDF_ENGINE_TENSOR)),
                                     None), b"only the FP32-unit engine"),
        (lambda: L.sdf_knn_mean_distance(None, 64, ctypes.byref(d), None), b"sdf_knn_mean_distance"),
        (lambda: L.sdf_paper_lambda(None, ctypes.byref(d), None, None), b"sdf_paper_lambda: NULL"),
        (lambda: L.sdf_cloud_info(None, ctypes.byref(i64), ctypes.byref(f), None, None), b"sdf_cloud_info: cloud"),
        (lambda: L.sdf_cloud_forms(None, ctypes.byref(i64), None), b"sdf_cloud_forms: cloud"),
        (lambda: L.sdf_build_weighted(fake, fake, fake, fake, 0, None, ctypes.byref(ctypes.c_void_p())),
         b"n must be"),
        (lambda: L.sdf_combine(7, fake, fake, 4, fake, None), b"sdf_combine: unknown op"),
        (lambda: L.sdf_combine(0, fake, fake, -1, fake, None), b"sdf_combine: q < 0"),
        (lambda: L.sdf_combine(0, None, fake, 4, fake, None), b"sdf_combine: NULL buffer"),
        (lambda: L.sdf_orient(fake, fake, fake, 1, 16, 3, ctypes.byref(o), ctypes.byref(i32), ctypes.byref(i32), None),
         b"sdf_orient: n must be"),
        (lambda: L.sdf_orient(fake, fake, fake, 100, 65, 3, ctypes.byref(o), ctypes.byref(i32), ctypes.byref(i32),
                              None), b"sdf_orient: k must be"),
        (lambda: L.sdf_orient(fake, fake, fake, 100, 16, 0, ctypes.byref(o), ctypes.byref(i32), ctypes.byref(i32),
                              None), b"sdf_orient: max_iter"),
        (lambda: L.sdf_mesh_level_set(fake, 1, 4, 4, one, one, 0.0, fake, 10, fake, 10, ctypes.byref(i64),
                                      ctypes.byref(i64), None), b"sdf_mesh_level_set: need at least 2"),
        (lambda: L.sdf_mesh_level_set(None, 4, 4, 4, one, one, 0.0, fake, 10, fake, 10, ctypes.byref(i64),
                                      ctypes.byref(i64), None), b"sdf_mesh_level_set: NULL"),
    ]


def test_every_entry_point_refuses_bad_arguments_on_the_host(abi):
    L = abi.lib()
    for call, msg in _refusals(abi):
        assert call() == abi.SDF_EINVAL, msg
        assert msg in L.sdf_last_error(), (msg, L.sdf_last_error())


def test_import_refuses_what_is_not_an_export(abi):
    """sdf_import checks the header and the size before any CUDA call."""
    import struct
    L = abi.lib()
    h = ctypes.c_void_p()
    n = 5
    good_size = 24 + n * (12 + 16) * 4 + n

    def blob(magic=b"PTSDFCK\0", version=1, weighted=0, count=n, size=good_size):
        head = magic + struct.pack("<IIq", version, weighted, count)
        return ctypes.create_string_buffer(head + b"\0" * (size - len(head)), size)

    cases = [(None, 100, b"buf or out is NULL"), (blob(), 10, b"shorter than the header"),
             (blob(magic=b"PTSDFCX\0"), good_size, b"not an sdf_export buffer"),
             (blob(version=2), good_size, b"not an sdf_export buffer"),
             (blob(weighted=3), good_size, b"not an sdf_export buffer"),
             (blob(count=0, size=24), 24, b"does not match its header"),
             (blob(), good_size - 1, b"does not match its header"),
             (blob(weighted=1), good_size, b"does not match its header")]
    for buf, size, msg in cases:
        assert L.sdf_import(buf, size, None, ctypes.byref(h)) == abi.SDF_EINVAL
        assert msg in L.sdf_last_error(), (msg, L.sdf_last_error())
    size = ctypes.c_int64()
    assert L.sdf_export(None, None, 0, ctypes.byref(size)) == abi.SDF_EINVAL
