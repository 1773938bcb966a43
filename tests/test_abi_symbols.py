"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point include/fitsne_gb300.h declares; host-only entry points behave as
documented (no device work is issued here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(tsne_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1712_09005_gb300 import build
    build.build()
    from paper_1712_09005_gb300 import _abi
    return _abi.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1712_09005_gb300 import _abi
    assert sorted(_abi.exported_names()) == declared_functions()


def test_host_only_entry_points(lib):
    from paper_1712_09005_gb300 import _abi
    assert lib.tsne_version().startswith(b"fitsne-gb300")
    sp = _abi.tsne_step_params()
    lib.tsne_step_params_default(ctypes.byref(sp))
    assert (sp.n_iter, sp.early_iters, sp.early_alpha, sp.lr) == (1000, 250, 12.0, 200.0)
    sp.late_iters, sp.late_alpha = 250, 4.0
    alphas = [lib.tsne_alpha_at(ctypes.byref(sp), i) for i in (0, 249, 250, 749, 750, 999)]
    assert alphas == [12.0, 12.0, 1.0, 1.0, 4.0, 4.0]


@pytest.mark.parametrize("N,s,n_int,p,n_int_max", [
    (1, 2, 0, 3, 0),       # N < 2
    (100, 3, 0, 3, 0),     # s not in {1, 2}
    (100, 2, 0, 1, 0),     # p < 2
    (100, 2, 0, 6, 0),     # p > 5
    (100, 2, 0, 3, 401),   # p * n_int_max > 1200 in 2-D
    (100, 1, 0, 3, 1001),  # p * n_int_max > 3000 in 1-D
    (100, 2, 500, 3, 0),   # fixed count above the cap
])
def test_plan_create_rejects_bad_arguments(lib, N, s, n_int, p, n_int_max):
    from paper_1712_09005_gb300 import _abi
    opts = _abi.tsne_plan_opts(0, n_int_max, None)
    out = ctypes.c_void_p(1)
    rc = lib.tsne_plan_create(N, s, n_int, p, ctypes.byref(opts), ctypes.byref(out))
    assert rc == _abi.TSNE_ERR_INVALID_ARG
    assert out.value is None
    assert lib.tsne_last_error_string()


def test_null_plan_is_rejected(lib):
    from paper_1712_09005_gb300 import _abi
    assert lib.tsne_plan_destroy(None) == 0
    assert lib.tsne_plan_status(None) == _abi.TSNE_ERR_INVALID_ARG
    assert lib.tsne_plan_launch_count(None) == 0


@pytest.mark.parametrize("N,D,k", [
    (100, 0, 10),      # D < 1
    (100, 65, 10),     # D > 64
    (100, 50, 0),      # k < 1
    (1000, 50, 257),   # k > 256
    (90, 50, 90),      # N <= k
    (1, 3, 1),         # N < 2
    (20_000_000, 50, 90),  # 2 N k above 2^31 - 1
])
def test_affinity_create_rejects_bad_arguments(lib, N, D, k):
    from paper_1712_09005_gb300 import _abi
    out = ctypes.c_void_p(1)
    rc = lib.tsne_affinity_create(N, D, k, None, ctypes.byref(out))
    assert rc == _abi.TSNE_ERR_INVALID_ARG
    assert out.value is None
    assert lib.tsne_last_error_string()


def test_null_affinity_is_rejected(lib):
    from paper_1712_09005_gb300 import _abi
    assert lib.tsne_affinity_destroy(None) == 0
    csr = _abi.tsne_csr()
    assert lib.tsne_affinity_compute(None, None, 30.0, ctypes.byref(csr)) == _abi.TSNE_ERR_INVALID_ARG
    assert lib.tsne_affinity_knn_copy(None, None, None, None) == _abi.TSNE_ERR_INVALID_ARG
    assert lib.tsne_affinity_launch_count(None) == 0


@pytest.mark.parametrize("n_bins,G,max_goi", [
    (0, 100, 4),              # no bins
    ((1 << 20) + 1, 100, 4),  # n_bins above 2^20
    (10, 0, 4),               # no genes
    (10, 100, 0),             # no genes of interest
    (10, 100, 65536),         # max_goi above 65535
    (1 << 20, 1 << 21, 1),    # n_bins x G above 2^40
])
def test_heatmap_create_rejects_bad_arguments(lib, n_bins, G, max_goi):
    from paper_1712_09005_gb300 import _abi
    out = ctypes.c_void_p(1)
    rc = lib.tsne_heatmap_create(n_bins, G, max_goi, None, ctypes.byref(out))
    assert rc == _abi.TSNE_ERR_INVALID_ARG
    assert out.value is None
    assert lib.tsne_last_error_string()


def test_null_heatmap_and_run_state_are_rejected(lib):
    from paper_1712_09005_gb300 import _abi
    assert lib.tsne_heatmap_destroy(None) == 0
    assert lib.tsne_heatmap_bin(None, None, 10, _abi.tsne_csr(), None, None) == _abi.TSNE_ERR_INVALID_ARG
    assert lib.tsne_heatmap_nearest(None, None, None, 1, 1, None, None) == _abi.TSNE_ERR_INVALID_ARG
    ms = (ctypes.c_double * 4)()
    assert lib.tsne_heatmap_phase_ms(None, ms) == _abi.TSNE_ERR_INVALID_ARG
    assert lib.tsne_heatmap_launch_count(None) == 0
    assert lib.tsne_run_state_save(None, None, None) == _abi.TSNE_ERR_INVALID_ARG
    assert lib.tsne_run_state_load(None, None, None) == _abi.TSNE_ERR_INVALID_ARG


@pytest.mark.parametrize("m,n,k,l", [
    (1, 100, 2, 4),      # m < 2
    (100, 102, 2, 4),    # n not a multiple of 4
    (100, 100, 0, 4),    # k < 1
    (100, 100, 5, 4),    # l < k
    (100, 100, 2, 65),   # l > 64
    (40, 100, 2, 40),    # l >= min(m, n)
])
def test_oocpca_create_rejects_bad_arguments(lib, m, n, k, l):
    from paper_1712_09005_gb300 import _abi
    out = ctypes.c_void_p()
    opts = _abi.tsne_oocpca_opts()
    rc = lib.tsne_oocpca_create(m, n, k, l, ctypes.byref(opts), ctypes.byref(out))
    assert rc == _abi.TSNE_ERR_INVALID_ARG
    assert not out.value
