"""The allocation-free symmetrisation entry point (ltsnet_symmetrize_static),
called through the C ABI.  It exists for callers that cannot allocate device
memory where they need this step (plug-ins and embedded hosts handed a fixed
device-memory budget that forbid allocation); it uses a scratch array built
into the library instead of a caller workspace.  Its
results must equal those of ltsnet_symmetrize, call after call (the scratch
array is reused and keeps the previous call's contents).

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _inputs(lt, g, u):
    k = int(np.ceil(3 * u - 1e-9))
    nbr, hop, cnt = lt.knn_bfs(g.row_ptr, g.col, k)
    beta, pcond, conv = lt.calibrate(hop, cnt, u)
    return nbr, cnt, pcond


def _static(lt, nbr, cnt, pcond):
    import torch

    n, k = nbr.shape
    L = lt.lib()
    cap = int(L.ltsnet_symmetrize_max_nnz(n, k))
    P_row = torch.empty((n + 1,), dtype=torch.int64, device="cuda")
    P_col = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    P_val = torch.full((cap,), -7.0, dtype=torch.float32, device="cuda")
    nnz = ctypes.c_int64(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.ltsnet_symmetrize_static(ctypes.c_void_p(nbr.data_ptr()), ctypes.c_void_p(cnt.data_ptr()),
                                    ctypes.c_void_p(pcond.data_ptr()), n, k, ctypes.c_void_p(P_row.data_ptr()),
                                    ctypes.c_void_p(P_col.data_ptr()), ctypes.c_void_p(P_val.data_ptr()), cap,
                                    ctypes.byref(nnz), stream)
    assert rc == 0, lt.status_string(rc)
    m = nnz.value
    return P_row.cpu().numpy(), P_col[:m].cpu().numpy(), P_val[:m].cpu().numpy()


def test_static_symmetrize_matches_workspace_version(ltlib):
    # the last case sits exactly at the limit: 2 n k = 2 * 2048 * 64 = 2^18
    cases = [(synth.grid2d(32, 32), 30.0), (synth.sbm([300, 250, 200], 12.0, 80, seed=8), 40.0),
             (synth.grid2d(64, 32), 64.0 / 3.0)]
    assert 2 * 2048 * 64 == ltlib.lib().ltsnet_symmetrize_static_max_entries()
    for g, u in cases:
        nbr, cnt, pcond = _inputs(ltlib, g, u)
        ref = [t.cpu().numpy() for t in ltlib.symmetrize(nbr, cnt, pcond)]
        for _ in range(2):  # two calls in a row reuse the same scratch array
            got = _static(ltlib, nbr, cnt, pcond)
            assert np.array_equal(got[0], ref[0])
            assert np.array_equal(got[1], ref[1])
            np.testing.assert_allclose(got[2], ref[2], rtol=1e-6, atol=0)


def test_static_symmetrize_rejects_oversized_input(ltlib):
    L = ltlib.lib()
    limit = int(L.ltsnet_symmetrize_static_max_entries())
    n, k = limit // 2 + 1, 1
    nnz = ctypes.c_int64(0)
    null = ctypes.c_void_p(0)
    rc = L.ltsnet_symmetrize_static(null, null, null, n, k, null, null, null, 0, ctypes.byref(nnz), null)
    assert rc == -2  # LTSNET_ERR_WORKSPACE, before any GPU work
