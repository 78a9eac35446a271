"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every function include/pwa.h declares; host-only queries and
argument validation behave as documented."""
import ctypes

import pytest

from paper_1108_5673_gb300 import _abi, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.load()


def test_exports_every_declared_symbol(lib):
    names = _abi.header_symbols()
    assert "pwa_nll_grad" in names and "pwa_build_norm" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_table_bytes_matches_paper_storage_estimate(lib):
    """Sec. 2: about 1.5 GB per million events for 20 waves (N^2 floats/event)."""
    b = _abi.pwa_table_bytes(20, 1_000_000)
    assert b == 20 * 20 * 4 * 1_000_000
    assert abs(b / 1.5e9 - 1) < 0.10
    with pytest.raises(_abi.PwaError):
        _abi.pwa_table_bytes(0, 10)


def test_version(lib):
    assert _abi.pwa_version() >= 100


def test_create_rejects_bad_config_before_touching_a_device(lib):
    for n_waves, max_k in ((0, 1), (49, 1), (4, 0)):
        cfg = _abi.pwa_config(n_waves, 0, 0, max_k, None)
        h = ctypes.c_void_p()
        rc = lib.pwa_create(ctypes.byref(h), 0, ctypes.byref(cfg))
        assert rc == _abi.PWA_EINVAL
        assert lib.pwa_last_error(None)
    assert lib.pwa_create(None, 0, None) == _abi.PWA_EINVAL


def test_null_context_is_rejected(lib):
    assert lib.pwa_nll(None, None, 1, None) == _abi.PWA_EINVAL
    assert lib.pwa_destroy(None) == _abi.PWA_OK
