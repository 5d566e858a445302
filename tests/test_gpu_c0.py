"""GPU parity of the preprocessing C0 (Alg. 3) against the FP64 oracle,
through the C ABI: partial BFS (bit-exact), beta search (FP64), symmetrisation
(integer structure bit-exact, values to FP32 rounding)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _graphs():
    iso = synth.csr_from_edges(40, np.array([0, 1, 2, 10, 11, 20]), np.array([1, 2, 3, 11, 12, 21]), "islands")
    star_u = np.zeros(300, np.int64)
    star_v = np.arange(1, 301)
    star = synth.csr_from_edges(301, np.concatenate([star_u, star_v[:-1]]), np.concatenate([star_v, star_v[1:]]),
                                "star+path")
    return [
        (synth.grid2d(32, 32), 90),
        (synth.grid2d(7, 5), 90),  # k > n - 1
        (synth.sbm([600, 500, 400, 300, 200], 12.0, 500, seed=11, name="sbm2000"), 120),
        (synth.random_recursive_tree(3000, 5), 90),
        (synth.barabasi_albert(3000, 4, seed=9), 150),
        (iso, 4),
        (star, 33),
        (synth.grid2d(20, 20), 1),
        (synth.grid2d(33, 31), 200),
    ]


def _bfs_both(lt, g, k):
    nbr, hop, cnt = lt.knn_bfs(g.row_ptr, g.col, k)
    rn, rh, rc = oracle.partial_bfs(g.row_ptr, g.col, k)
    return (nbr.cpu().numpy(), hop.cpu().numpy().astype(np.int32), cnt.cpu().numpy()), (rn, rh, rc)


@pytest.mark.parametrize("case", range(9))
def test_bfs_bit_exact(ltlib, case):
    g, k = _graphs()[case]
    (nbr, hop, cnt), (rn, rh, rc) = _bfs_both(ltlib, g, k)
    assert np.array_equal(cnt, rc)
    assert np.array_equal(nbr, rn)
    assert np.array_equal(hop, rh)


def test_bfs_rgg_1m_sampled_sources(ltlib):
    """Full-size random geometric graph (n ~ 1e6, k = 90): every row from the
    GPU run, checked bit for bit against the oracle on 4000 sampled sources."""
    g = synth.rgg()
    k = 90
    nbr, hop, cnt = ltlib.knn_bfs(g.row_ptr, g.col, k)
    nbr, hop, cnt = nbr.cpu().numpy(), hop.cpu().numpy().astype(np.int32), cnt.cpu().numpy()
    rng = np.random.default_rng(1)
    for s in np.sort(rng.choice(g.n, 4000, replace=False)):
        rn, rh, rc = oracle.partial_bfs(g.row_ptr, g.col, k, int(s), int(s) + 1)
        assert cnt[s] == rc[0]
        assert np.array_equal(nbr[s], rn[0]) and np.array_equal(hop[s], rh[0])


def _calib_check(beta, pcond, conv, rb, rp, rc, hop, cnt, u, tol):
    # The search takes the same steps on both sides; a row may differ only if
    # the oracle's |H - ln u| sits within rounding of the tolerance.
    same = beta == rb
    if not np.all(same):
        bad = np.flatnonzero(~same)
        for i in bad:
            c = cnt[i]
            d2 = hop[i, :c].astype(np.float64) ** 2
            w = np.exp(-rb[i] * (d2 - d2.min()))
            p = w / w.sum()
            H = -np.sum(p[p > 0] * np.log(p[p > 0]))
            assert abs(abs(H - np.log(u)) - tol) < 1e-12, f"row {i}: beta {beta[i]} vs {rb[i]}"
    ok = same
    assert np.array_equal(conv[ok], rc[ok])
    np.testing.assert_allclose(pcond[ok], rp[ok], rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("case,u", [(0, 30.0), (2, 40.0), (3, 30.0), (4, 50.0), (5, 1.3), (6, 11.0), (8, 66.7)])
def test_calibrate(ltlib, case, u):
    g, _ = _graphs()[case]
    k = oracle.k_from_perplexity(u)
    nbr, hop, cnt = ltlib.knn_bfs(g.row_ptr, g.col, k)
    beta, pcond, conv = ltlib.calibrate(hop, cnt, u)
    h = hop.cpu().numpy().astype(np.int32)
    c = cnt.cpu().numpy()
    rb, rp, rc = oracle.calibrate(h, c, u)
    _calib_check(beta.cpu().numpy(), pcond.cpu().numpy(), conv.cpu().numpy(), rb, rp, rc, h, c, u, 1e-5)


def test_calibrate_many_shells(ltlib):
    """A path graph gives one shell per hop (more than the kernel keeps in
    shared memory), exercising the per-neighbour fallback."""
    n = 400
    g = synth.csr_from_edges(n, np.arange(n - 1), np.arange(1, n))
    u = 60.0
    k = oracle.k_from_perplexity(u)
    nbr, hop, cnt = ltlib.knn_bfs(g.row_ptr, g.col, k)
    beta, pcond, conv = ltlib.calibrate(hop, cnt, u)
    h = hop.cpu().numpy().astype(np.int32)
    c = cnt.cpu().numpy()
    rb, rp, rc = oracle.calibrate(h, c, u)
    _calib_check(beta.cpu().numpy(), pcond.cpu().numpy(), conv.cpu().numpy(), rb, rp, rc, h, c, u, 1e-5)


@pytest.mark.parametrize("case,u", [(0, 30.0), (2, 40.0), (4, 50.0), (5, 1.3), (6, 11.0), (1, 30.0)])
def test_symmetrize(ltlib, case, u):
    g, _ = _graphs()[case]
    aff = ltlib.affinities(g.row_ptr, g.col, u)
    P_row, P_col, P_val = (t.cpu().numpy() for t in aff["P"])
    # the oracle symmetrises the GPU's own conditional rows, so any
    # difference is the symmetrisation's
    nbr = aff["nbr"].cpu().numpy()
    cnt = aff["cnt"].cpu().numpy()
    pc = aff["pcond"].cpu().numpy()
    rr, rc, rv = oracle.symmetrize(nbr, cnt, pc)
    assert np.array_equal(P_row, rr)
    assert np.array_equal(P_col, rc)
    assert np.array_equal(P_val, rv.astype(np.float32))


def test_preprocess_sbm100k(ltlib):
    """Power-law SBM, n = 1e5, u = 40: the whole C0 against the oracle's."""
    g = synth.sbm_powerlaw()
    u = 40.0
    aff = ltlib.affinities(g.row_ptr, g.col, u)
    ref = oracle.preprocess(g.row_ptr, g.col, u)
    assert np.array_equal(aff["nbr"].cpu().numpy(), ref.nbr)
    assert np.array_equal(aff["hop"].cpu().numpy().astype(np.int32), ref.hop)
    P_row, P_col, P_val = (t.cpu().numpy() for t in aff["P"])
    assert np.array_equal(P_row, ref.P_row)
    assert np.array_equal(P_col, ref.P_col)
    rel = np.abs(P_val.astype(np.float64) - ref.P_val64) / ref.P_val64
    assert rel.max() < 1.2e-7  # one FP32 rounding
    assert abs(P_val.astype(np.float64).sum() - 1.0) < 1e-5
