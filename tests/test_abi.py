"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/ltsnet.h; host-only calls behave as documented."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2509_19785_gb300 as lt

    return lt


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ltsnet.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(ltsnet_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("ltsnet_knn_bfs", "ltsnet_calibrate", "ltsnet_symmetrize", "ltsnet_gradient", "ltsnet_optimize",
                 "ltsnet_run", "ltsnet_run_host"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\bT (ltsnet_[a-z0-9_]+)", out.stdout))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(lib.ABI_SYMBOLS) <= set(declared_functions())


def test_default_params_and_stages(lib):
    p = lib.lib().ltsnet_default_params()
    assert p.perplexity == 30.0 and abs(p.eps - 0.05) < 1e-9 and p.nodes_per_box == 3
    assert p.n_stages == 2 and p.stages[0].iters == 250 and p.stages[1].iters == 750
    st = lib.default_stages(100)
    assert len(st) == 1 and st[0].iters == 100
    st = lib.default_stages(1000)
    assert [s.iters for s in st] == [250, 750] and abs(st[1].lambda_r - 0.6) < 1e-6


def test_status_strings(lib):
    for code in (0, 1, -1, -2, -3, -4, -5, -6):
        assert lib.status_string(code) and "unknown" not in lib.status_string(code)
    assert "unknown" in lib.status_string(42)


def test_workspace_sizes_and_argument_checks(lib):
    L = lib.lib()
    cp = lib.Params().to_c()
    assert L.ltsnet_gradient_workspace_size(1000, ctypes.byref(cp)) > 0
    assert L.ltsnet_run_workspace_size(1000, 4000, ctypes.byref(cp)) > L.ltsnet_gradient_workspace_size(
        1000, ctypes.byref(cp))
    assert L.ltsnet_symmetrize_max_nnz(10, 3) == 60
    bad = lib.Params(nodes_per_box=7).to_c()
    assert L.ltsnet_gradient_workspace_size(1000, ctypes.byref(bad)) == 0
    big = lib.Params(max_boxes=5000).to_c()
    assert L.ltsnet_gradient_workspace_size(1000, ctypes.byref(big)) == 0
    # argument errors are caught on the host before any CUDA call
    null = ctypes.c_void_p(0)
    assert L.ltsnet_knn_bfs(null, null, 10, 0, null, null, null, null, 0, null) == -1
    assert L.ltsnet_knn_bfs(null, null, 10, 5000, null, null, null, null, 0, null) == -1
    assert L.ltsnet_calibrate(null, null, 10, 3, -1.0, 1e-5, 10, null, null, null, null) == -1
    assert L.ltsnet_gradient(null, null, null, 10, null, None, ctypes.byref(cp), null, null, null, null, 0,
                             null) == -1


def test_calls_beside_the_path_check_arguments_on_the_host(lib):
    """Pivot MDS, the quadtree variants and the quality metrics: workspace
    sizes without a GPU, and argument errors returned before any CUDA call."""
    L = lib.lib()
    cp = lib.Params().to_c()
    null = ctypes.c_void_p(0)
    one = ctypes.c_void_p(256)  # never dereferenced: every call below fails its checks first
    # Pivot MDS: 2 <= k <= min(n, 512); grows with n and k
    assert L.ltsnet_pivot_mds_workspace_size(1000, 100) > L.ltsnet_pivot_mds_workspace_size(1000, 10) > 0
    assert L.ltsnet_pivot_mds_workspace_size(2000, 10) > L.ltsnet_pivot_mds_workspace_size(1000, 10)
    for n, k in ((1000, 1), (1000, 513), (10, 11), (1, 1)):
        assert L.ltsnet_pivot_mds_workspace_size(n, k) == 0
    eig = (ctypes.c_double * 2)()
    for n, k, first in ((10, 1, 0), (10, 11, 0), (10, 4, -1), (10, 4, 10)):
        assert L.ltsnet_pivot_mds(one, one, n, k, first, 1e-4, one, one, null, eig, one, 1 << 30, null) == -1
    assert L.ltsnet_pivot_mds(one, one, 10, 4, 0, -1.0, one, one, null, eig, one, 1 << 30, null) == -1
    # a workspace that is too small or misaligned
    need = L.ltsnet_pivot_mds_workspace_size(10, 4)
    assert L.ltsnet_pivot_mds(one, one, 10, 4, 0, 1e-4, one, one, null, eig, one, need - 1, null) == -2
    assert L.ltsnet_pivot_mds(one, one, 10, 4, 0, 1e-4, one, one, null, eig, ctypes.c_void_p(257), need,
                              null) == -2
    # quadtree gradient and loop: variant 1 (BH) or 2 (FIt), theta >= 0
    assert L.ltsnet_gradient_quadtree_workspace_size(1000, ctypes.byref(cp), 1) > 0
    assert L.ltsnet_gradient_quadtree_workspace_size(1000, ctypes.byref(cp), 2) > \
        L.ltsnet_gradient_quadtree_workspace_size(1000, ctypes.byref(cp), 1)
    assert L.ltsnet_gradient_quadtree_workspace_size(1000, ctypes.byref(cp), 3) == 0
    st = lib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8).to_c()
    terms = (ctypes.c_double * 2)()
    for theta, variant in ((-0.5, 1), (0.5, 0), (float("nan"), 1)):
        assert L.ltsnet_gradient_quadtree(one, one, one, 100, one, ctypes.byref(st), ctypes.byref(cp), theta,
                                          variant, one, null, terms, one, 1 << 30, null) == -1
    assert L.ltsnet_optimize_quadtree_workspace_size(1000, ctypes.byref(cp), 1) > \
        L.ltsnet_gradient_quadtree_workspace_size(1000, ctypes.byref(cp), 1)
    assert L.ltsnet_optimize_quadtree(one, one, one, 100, ctypes.byref(cp), 0.5, 1, one, one, one, -1, 5, one,
                                      1 << 30, null) == -1
    # quality metrics
    assert L.ltsnet_quality_workspace_size(1000, 4000) > 0 and L.ltsnet_quality_workspace_size(0, 0) == 0
    assert L.ltsnet_quality_workspace_size(1000, 400000) > L.ltsnet_quality_workspace_size(1000, 4000)
    npv = ctypes.c_double()
    assert L.ltsnet_neighbourhood_preservation(one, one, 0, one, null, null, ctypes.byref(npv), one, 1 << 30,
                                               null) == -1
    out = (ctypes.c_double * 4)()
    assert L.ltsnet_stress(one, one, 10, one, one, 0, out, one, 1 << 30, null) == -1
    assert L.ltsnet_stress(one, one, 10, one, one, 3, out, one, 16, null) == -2


def test_every_entry_point_cites_the_paper_or_says_it_has_no_counterpart():
    """Each declaration in include/ltsnet.h is governed by a block comment
    (the closest one above it that is not a trailing comment of a #define)
    that cites the passage defining the operation (Sec., Eq., Alg.) or says
    that the call has no counterpart in the paper."""
    text = open(os.path.join(ROOT, "include", "ltsnet.h")).read()
    blocks = [(m.start(), m.end(), m.group(0)) for m in re.finditer(r"/\*.*?\*/", text, flags=re.S)
              if not text[text.rfind("\n", 0, m.start()) + 1:m.start()].lstrip().startswith("#define")]
    cite = re.compile(r"Sec\.|Eq\.|Alg\.|no counterpart|not part of the method", re.I)
    for name in declared_functions():
        pos = re.search(r"\b" + name + r"\s*\(", re.sub(r"/\*.*?\*/", lambda m: " " * len(m.group(0)), text,
                                                        flags=re.S)).start()
        above = [b for b in blocks if b[1] <= pos]
        assert above, name
        assert cite.search(above[-1][2]), name


def test_static_symmetrize_size_check_at_the_limit(lib):
    """The allocation-free symmetrisation accepts every shape with
    2 n k = ltsnet_symmetrize_static_max_entries() (its built-in scratch
    holds that call's workspace) and rejects one more entry with
    LTSNET_ERR_WORKSPACE, on the host.  Null buffers make an accepted call stop
    at its next check (an argument error, or a CUDA error where there is no
    GPU), never at the size check."""
    L = lib.lib()
    limit = int(L.ltsnet_symmetrize_static_max_entries())
    null = ctypes.c_void_p(0)
    nnz = ctypes.c_int64(0)
    k = 1
    while k <= 4096:
        n = limit // (2 * k)
        assert 2 * n * k == limit
        assert L.ltsnet_symmetrize_workspace_size(n, k) > 0
        rc = L.ltsnet_symmetrize_static(null, null, null, n, k, null, null, null, 0, ctypes.byref(nnz), null)
        assert rc in (-1, -3), (n, k, rc)
        rc = L.ltsnet_symmetrize_static(null, null, null, n + 1, k, null, null, null, 0, ctypes.byref(nnz), null)
        assert rc == -2, (n + 1, k, rc)
        k *= 2
