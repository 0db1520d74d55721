"""The C-ABI library builds for sm_103a, loads, and exports every function the
header declares; host-side argument checks reject bad calls without touching a
GPU.  No kernel is launched here."""
import ctypes
import shutil

import numpy as np
import pytest

from paper_1504_06474_gb300 import _build
from paper_1504_06474_gb300 import ssspmv as S

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not
                                __import__("os").path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return S._lib()


def test_exports_every_declared_function(lib):
    names = S.declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    # and the binding wraps each of them under the same name
    for n in names:
        assert callable(getattr(S, n)), n


def test_host_only_queries(lib):
    assert S.ssspmv_version() >= 10000
    assert S.ssspmv_strerror(S.SSSPMV_EINVAL) == "invalid argument"
    ws = S.ssspmv_supported_w()
    assert ws and all(w % 2 == 1 and w <= 31 for w in ws)
    # workspace size does not depend on a device
    a = S.ssspmv_workspace_bytes(4_096_000, 109_215_352, 8, None)
    b = S.ssspmv_workspace_bytes(4_096_000, 109_215_352, 8, S.make_opts(W=27))
    assert a > 0 and b > 0 and a % 256 == 0
    assert S.ssspmv_workspace_bytes(-1, 0, 8, None) == 0
    assert S.ssspmv_workspace_bytes(10, 10, 8, S.make_opts(W=4)) == 0  # even W not compiled
    assert S.ssspmv_workspace_bytes(10, 10, 3, None) == 0


def test_default_shape_rules(lib):
    """The defaults chosen on the host: tiles per bunch S = ceil(ntiles/32768)
    up to 4, and the tile width (the shortest, but 27 for BF16 values when
    rows hold 20 entries or more on average); the workspace is sized for the
    same S, so it never depends on the device."""
    sh = S.ssspmv_plan_shape
    for ntiles, want in ((1, 1), (130, 1), (32768, 1), (32769, 2), (65536, 2), (98304, 3),
                         (98305, 4), (227_532, 4)):
        got = sh(4096, ntiles * 480, 8, None)
        assert (got["W"], got["ntiles"], got["S"]) == (15, ntiles, want), (ntiles, got)
        assert got["nbunches"] == -(-ntiles // want)
    assert sh(4096, 62_167, 8, S.make_opts(S=4))["S"] == 4  # an explicit S stands
    # tile width: BF16 values with long rows, everything else the shortest
    assert sh(4_096_000, 109_215_352, 2, None)["W"] == 27     # stencil, 26.7 per row
    assert sh(4_194_304, 66_242_182, 2, None)["W"] == 15      # R-MAT, 15.8 per row
    assert sh(1000, 19_999, 2, None)["W"] == 15 and sh(1000, 20_000, 2, None)["W"] == 27
    for vb in (8, 4):
        assert sh(4_096_000, 109_215_352, vb, None)["W"] == 15
    assert sh(4_096_000, 109_215_352, 2, S.make_opts(W=21))["W"] == 21


FAKE = 0x7f0000000000  # never dereferenced: every call below fails on the host


@pytest.mark.parametrize("args,code", [
    ((-1, 4, 0), S.SSSPMV_EINVAL),
    ((4, -1, 0), S.SSSPMV_EINVAL),
    ((0, 4, 3), S.SSSPMV_EINVAL),
])
def test_bad_scalars(lib, args, code):
    m, n, nnz = args
    rc = S.ssspmv_csr_f64(m, n, nnz, FAKE, FAKE, FAKE, FAKE, FAKE, workspace=FAKE, ws_bytes=1 << 30)
    assert rc == code


def test_null_and_misaligned(lib):
    rc = S.ssspmv_csr_f64(4, 4, 8, None, FAKE, FAKE, FAKE, FAKE, workspace=FAKE, ws_bytes=1 << 30)
    assert rc == S.SSSPMV_EINVAL
    rc = S.ssspmv_csr_f64(4, 4, 8, FAKE, FAKE + 4, FAKE, FAKE, FAKE, workspace=FAKE,
                          ws_bytes=1 << 30)
    assert rc == S.SSSPMV_EINVAL          # col_idx not 16-byte aligned
    rc = S.ssspmv_csr_f64(4, 4, 8, FAKE, FAKE, FAKE + 8, FAKE, FAKE, workspace=FAKE,
                          ws_bytes=1 << 30)
    assert rc == S.SSSPMV_EINVAL          # val not 16-byte aligned
    rc = S.ssspmv_csr_f64(4, 0, 8, FAKE, FAKE, FAKE, FAKE, FAKE, workspace=FAKE, ws_bytes=1 << 30)
    assert rc == S.SSSPMV_EINVAL          # entries but no columns


def test_workspace_checks(lib):
    need = S.ssspmv_workspace_bytes(100, 1000, 8, None)
    # workspace=None asks for the library-owned buffer; with no GPU here the
    # device lookup fails before anything is allocated or launched
    rc = S.ssspmv_csr_f64(100, 100, 1000, FAKE, FAKE, FAKE, FAKE, FAKE, workspace=None,
                          ws_bytes=need)
    assert rc == S.SSSPMV_ECUDA
    # the debug entry point reads its artefacts back from the workspace: it needs one
    rc = S._lib().ssspmv_csr_f64_debug(100, 100, 1000, FAKE, FAKE, FAKE, FAKE, FAKE, None, None,
                                       0, None, None, None, None, None, None)
    assert rc == S.SSSPMV_EWORKSPACE
    rc = S.ssspmv_csr_f64(100, 100, 1000, FAKE, FAKE, FAKE, FAKE, FAKE, workspace=FAKE,
                          ws_bytes=need - 1)
    assert rc == S.SSSPMV_EWORKSPACE
    rc = S.ssspmv_csr_f64(100, 100, 1000, FAKE, FAKE, FAKE, FAKE, FAKE, workspace=FAKE + 16,
                          ws_bytes=need)
    assert rc == S.SSSPMV_EWORKSPACE      # workspace must be 256-byte aligned


def test_bad_opts(lib):
    o = S.make_opts(S=-3)
    rc = S.ssspmv_csr_f64(4, 4, 8, FAKE, FAKE, FAKE, FAKE, FAKE, opts=o, workspace=FAKE,
                          ws_bytes=1 << 30)
    assert rc == S.SSSPMV_EINVAL
    o = S.make_opts(W=16)
    rc = S.ssspmv_csr_f64(4, 4, 8, FAKE, FAKE, FAKE, FAKE, FAKE, opts=o, workspace=FAKE,
                          ws_bytes=1 << 30)
    assert rc == S.SSSPMV_EUNSUPPORTED


def test_empty_matrix_is_a_noop(lib):
    # m == 0: nothing to write, nothing launched
    assert S.ssspmv_csr_f64(0, 5, 0, None, None, None, None, None) == S.SSSPMV_OK


def test_opts_struct_layout(lib):
    assert ctypes.sizeof(S.ssspmv_opts) == 24
    assert S.ssspmv_opts.timer.offset == 16


def test_torch_layer_imports(lib):
    pytest.importorskip("torch")
    from paper_1504_06474_gb300 import api, ssspmv
    assert callable(api.spmv_f64) and callable(api.spmv_f64_debug)
    assert api._c is ssspmv


def test_plan_host_checks(lib):
    import ctypes
    h = ctypes.c_void_p()
    L = S._lib()
    # bad scalars, missing row_ptr, unknown value type, no output handle
    assert L.ssspmv_plan_create(-1, 4, 0, FAKE, 8, None, None, 0, None, ctypes.byref(h)) == S.SSSPMV_EINVAL
    assert L.ssspmv_plan_create(0, 4, 3, FAKE, 8, None, None, 0, None, ctypes.byref(h)) == S.SSSPMV_EINVAL
    assert L.ssspmv_plan_create(4, 4, 8, None, 8, None, None, 0, None, ctypes.byref(h)) == S.SSSPMV_EINVAL
    assert L.ssspmv_plan_create(4, 4, 8, FAKE, 3, None, None, 0, None, ctypes.byref(h)) == S.SSSPMV_EUNSUPPORTED
    assert L.ssspmv_plan_create(4, 4, 8, FAKE, 8, None, None, 0, None, None) == S.SSSPMV_EINVAL
    # a timer belongs to executions, not to the plan
    o = S.make_opts(timer=12345)
    assert L.ssspmv_plan_create(4, 4, 8, FAKE, 8, ctypes.byref(o), None, 0, None,
                                ctypes.byref(h)) == S.SSSPMV_EINVAL
    # a caller workspace that is too small or misaligned is refused before any launch
    need = S.ssspmv_workspace_bytes(100, 1000, 8, None)
    assert L.ssspmv_plan_create(100, 100, 1000, FAKE, 8, None, FAKE, need - 1, None,
                                ctypes.byref(h)) == S.SSSPMV_EWORKSPACE
    assert L.ssspmv_plan_create(100, 100, 1000, FAKE, 8, None, FAKE + 16, need, None,
                                ctypes.byref(h)) == S.SSSPMV_EWORKSPACE
    assert h.value is None
    assert L.ssspmv_plan_execute(None, FAKE, FAKE, FAKE, FAKE, None, None) == S.SSSPMV_EINVAL
    S.ssspmv_plan_destroy(None)  # a no-op


def test_rows_variant_host_checks(lib):
    o = S.make_opts(W=3, variant=S.VARIANT_ROWS)        # lanes per row: a power of two <= 32
    assert S.ssspmv_csr_f64(4, 4, 8, FAKE, FAKE, FAKE, FAKE, FAKE, opts=o, workspace=FAKE,
                            ws_bytes=1 << 30) == S.SSSPMV_EINVAL
    o = S.make_opts(W=8, variant=S.VARIANT_ROWS)
    assert S.ssspmv_workspace_bytes(100, 1000, 8, o) > 0
    assert S.ssspmv_plan_shape(100, 1000, 8, o)["W"] == 8
    # FP64 single calls only
    assert S.ssspmv_csr_f32(4, 4, 8, FAKE, FAKE, FAKE, FAKE, FAKE, opts=o, workspace=FAKE,
                            ws_bytes=1 << 30) == S.SSSPMV_EUNSUPPORTED
    assert S.ssspmv_batched_workspace_bytes(3, 1000, 4, o) == 0
    import ctypes
    h = ctypes.c_void_p()
    assert S._lib().ssspmv_plan_create(4, 4, 8, FAKE, 8, ctypes.byref(o), None, 0, None,
                                       ctypes.byref(h)) == S.SSSPMV_EUNSUPPORTED


def test_batched_and_axpby_host_checks(lib):
    # batches: bad counts and bounds, missing or misaligned descriptor array, workspace
    assert S.ssspmv_batched_workspace_bytes(-1, 100, 4, None) == 0
    assert S.ssspmv_batched_workspace_bytes(3, -5, 4, None) == 0
    assert S.ssspmv_batched_workspace_bytes(3, 100, 8, None) == 0        # FP32 only
    need = S.ssspmv_batched_workspace_bytes(3, 1000, 4, None)
    assert need > 0
    L = S._lib()
    assert L.ssspmv_csr_batched_f32(0, None, 0, None, None, 0, None) == S.SSSPMV_OK  # nothing
    assert L.ssspmv_csr_batched_f32(3, None, 1000, None, FAKE, need, None) == S.SSSPMV_EINVAL
    assert L.ssspmv_csr_batched_f32(3, FAKE + 4, 1000, None, FAKE, need, None) == S.SSSPMV_EINVAL
    assert L.ssspmv_csr_batched_f32(3, FAKE, 1000, None, FAKE, need - 1, None) == S.SSSPMV_EWORKSPACE
    assert L.ssspmv_csr_batched_f32(3, FAKE, 1000, None, FAKE + 16, need, None) == S.SSSPMV_EWORKSPACE
    # y = alpha A x + beta y: the same argument checks as the plain call
    assert S.ssspmv_csr_f64_axpby(-1, 4, 8, FAKE, FAKE, FAKE, FAKE, FAKE, 1.0, 0.0, workspace=FAKE,
                                  ws_bytes=1 << 30) == S.SSSPMV_EINVAL
    assert S.ssspmv_csr_f64_axpby(4, 4, 8, FAKE, FAKE, FAKE + 8, FAKE, FAKE, 1.0, 0.0,
                                  workspace=FAKE, ws_bytes=1 << 30) == S.SSSPMV_EINVAL
    assert L.ssspmv_plan_execute_axpby(None, FAKE, FAKE, FAKE, FAKE, 1.0, 0.0, None, None) == \
        S.SSSPMV_EINVAL


def test_selector_host_side(lib):
    from paper_1504_06474_gb300 import selector as sel
    assert sel.K == len(sel.CLASSES) and sel.CLASSES[0][1] == {}          # class 0: defaults
    assert S.ssspmv_mlp_param_count(16, 64, 64, sel.K) == \
        16 * 64 + 64 + 64 * 64 + 64 + sel.K * 64 + sel.K
    assert S.ssspmv_mlp_param_count(0, 64, 64, 10) == 0
    p = sel.load_default()                                                  # shipped weights
    assert p is not None and p.size == S.ssspmv_mlp_param_count(16, 64, 64, sel.K)
    t = np.array([[2.0, 1.0, 3.0], [1.0, 1.0, 1.0]])
    r = sel.evaluate(np.array([1, 2]), t)
    assert r["mean_regret"] == 0.0 and r["optimum_hit_rate"] == 1.0
    assert np.isclose(r["geomean_speedup_vs_default"], np.sqrt(2.0))
    specs = sel.dataset_specs(50, seed=9)
    assert specs == sel.dataset_specs(50, seed=9)
    assert {sp[0] for sp in specs} <= set(sel.FAMILIES)
