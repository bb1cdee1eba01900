"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against what the paper and the mathematics fix:
an independent library (cuRAND's host Philox, mpmath, scipy), closed forms
(tests/golden/), derivative identities by finite differences, brute force on
tiny graphs, and invariants of Fig. 2 / Fig. 4.  None of them calls the CUDA
engine.
"""
import ctypes
import math
import os

import mpmath as mp
import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
MU = 1.5


# ---------------------------------------------------------------------------
# Philox4x32-10 against cuRAND's host generator (an independent implementation)
# ---------------------------------------------------------------------------
def _curand_host(seed, count, offset=0):
    path = None
    for cand in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            lib = ctypes.CDLL(cand)
            path = cand
            break
        except OSError:
            continue
    if path is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    if offset:
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
    out = np.zeros(count, dtype=np.uint32)
    assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
    lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x6E6D7065, (0xDEADBEEF << 32) | 0x12345678])
def test_philox_matches_curand_host(oracle_mod, seed):
    # cuRAND's host Philox emits block b as Philox(ctr=(0,0,b,0), key=(seed_lo, seed_hi));
    # a small generator offset of 4*b words starts at block b.  Counter words 0, 1 and 3
    # stay zero only in the first round: rounds 2-10 mix every word, so the whole round
    # function and key schedule are exercised.
    key = [seed & 0xFFFFFFFF, seed >> 32]
    out = _curand_host(seed, 4 * 64)
    for b in range(64):
        np.testing.assert_array_equal(oracle_mod.philox4x32_10([0, 0, b, 0], key), out[4 * b: 4 * b + 4])
    for blk in (1000, 12345, 40000):
        got = _curand_host(seed, 8, offset=4 * blk)
        ctr = [0, 0, blk & 0xFFFFFFFF, blk >> 32]
        np.testing.assert_array_equal(oracle_mod.philox4x32_10(ctr, key), got[:4])


def test_philox_counter_words_all_matter(oracle_mod):
    base = oracle_mod.philox4x32_10([1, 2, 3, 4], [5, 6])
    for w in range(4):
        c = [1, 2, 3, 4]
        c[w] ^= 1
        assert not np.array_equal(oracle_mod.philox4x32_10(c, [5, 6]), base)


def test_vertex_draws_uniform(oracle_mod, sbm_small):
    # chi-square on the mapped draws of an empty-ish graph: every vertex equally likely
    n = 97
    rp = np.zeros(n + 1, dtype=np.int32)
    ci = np.zeros(0, dtype=np.int32)
    s = oracle_mod.sample(rp, ci, epoch=3, seed=99, k=200, max_retries=1)
    counts = np.zeros(n)
    for i in range(n):
        row = s[i][s[i] >= 0]
        assert np.all(row != i)
        np.add.at(counts, row, 1)
    # self draws are rejected (max_retries=1) so vertex j receives draws from n-1 anchors
    draws = (s >= 0).sum()
    expected = draws / n
    chi2 = ((counts - expected) ** 2 / expected).sum()
    from scipy.stats import chi2 as chi2d
    assert chi2d.sf(chi2, n - 1) > 1e-4


def test_init_positions_exact_grid(oracle_mod):
    x = oracle_mod.init_positions(500, 3, seed=11)
    assert x.dtype == np.float32 and x.shape == (500, 3)
    assert x.min() >= -1.0 and x.max() < 1.0
    # values are k * 2^-23 - 1: exactly representable, no rounding happened
    k = (x.astype(np.float64) + 1.0) * 2 ** 23
    np.testing.assert_array_equal(k, np.round(k))
    assert abs(x.mean()) < 0.05
    x2 = oracle_mod.init_positions(500, 3, seed=11, init_range=0.25)
    np.testing.assert_array_equal(x2, (x.astype(np.float64) * 0.25).astype(np.float32))


# ---------------------------------------------------------------------------
# Membership
# ---------------------------------------------------------------------------
def test_membership_all_pairs(oracle_mod, sbm_small):
    rp, ci = sbm_small
    n = len(rp) - 1
    dense = np.zeros((n, n), dtype=bool)
    for i in range(n):
        dense[i, ci[rp[i]:rp[i + 1]]] = True
    assert np.array_equal(dense, dense.T) and not dense.diagonal().any()
    for i in range(n):
        for j in range(n):
            assert oracle_mod.is_edge(rp, ci, i, j) == dense[i, j]


# ---------------------------------------------------------------------------
# Description length (Sec. II.B) against mpmath
# ---------------------------------------------------------------------------
def _mp_dl(delta, mu, sigma, edge):
    # evaluated at the caller's working precision (see _mp)
    x = (mp.mpf(delta) - mu) / (mp.sqrt(2) * sigma)
    # 1/2 -/+ 1/2 erf(x) written as 1/2 erfc(+/-x); when that is close to 1 the
    # logarithm is taken as log1p of minus the other tail, exact in any precision
    a = x if edge else -x
    if a < 0:
        return -mp.log1p(-mp.erfc(-a) / 2) / mp.log(2)
    return -mp.log(mp.erfc(a) / 2, 2)


@pytest.mark.parametrize("sigma", [0.05, 0.3, 1.0, 2.5])
def test_dl_matches_mpmath(oracle_mod, sigma):
    for delta in [0.0, 0.01, 0.5, 1.2, 1.5, 1.9, 3.0, 7.5, 20.0]:
        for edge in (True, False):
            with mp.workdps(60):
                ref = float(_mp_dl(delta, MU, sigma, edge))
            got = oracle_mod.dl(delta, MU, sigma, edge)
            assert got == pytest.approx(ref, rel=1e-12, abs=1e-300), (delta, sigma, edge)


def test_h_basic_closed_forms(oracle_mod):
    n = 101
    N = n * (n - 1) / 2
    assert oracle_mod.h_basic(n, N / 2) == pytest.approx(1.0, abs=1e-15)
    assert oracle_mod.h_basic(n, 0) == 0.0
    assert oracle_mod.h_basic(n, N) == 0.0
    assert oracle_mod.h_basic(n, N / 4) == pytest.approx(oracle_mod.h_basic(n, 3 * N / 4), rel=1e-14)
    p = 0.1
    assert oracle_mod.h_basic(n, p * N) == pytest.approx(-(p * math.log2(p) + (1 - p) * math.log2(1 - p)))


# ---------------------------------------------------------------------------
# Parabola (Eq. 4 / Eq. 5)
# ---------------------------------------------------------------------------
def test_parabola_golden_closed_forms(oracle_mod):
    path = os.path.join(HERE, "golden", "parabola_closed_forms.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert rows
    for reading, kind, mu, sigma, w, d in rows:
        dd, ww = oracle_mod.parabola(float(mu), float(mu), float(sigma), kind == "edge",
                                     w_formula=(reading == "printed"), clamp_neg_d=0)
        assert ww == pytest.approx(float(w), rel=1e-13)
        assert dd == pytest.approx(float(d), rel=1e-13)


def _mp_derivs(delta, mu, sigma, edge):
    with mp.workdps(80):
        f = lambda t: _mp_dl(t, mu, sigma, edge)
        return mp.diff(f, mp.mpf(delta), 1), mp.diff(f, mp.mpf(delta), 2)


@pytest.mark.parametrize("sigma", [0.1, 0.7, 1.0, 3.0])
def test_parabola_matches_dl_derivatives(oracle_mod, sigma):
    """Sec. II.C: the parabola w(delta-d)^2 agrees with dl in the first and
    second derivative at the current distance (derived reading); the printed
    Eq. 4 agrees in the first derivative only."""
    deltas = [0.0, 0.2, 0.9, 1.5, 2.2, 4.0]
    deltas += [MU + sigma * u for u in (-30.0, -8.0, 6.0, 27.0, 40.0)]   # tail branches
    for delta in deltas:
        if delta < 0:
            continue
        for edge in (True, False):
            d1, d2 = _mp_derivs(delta, MU, sigma, edge)
            d1, d2 = float(d1), float(d2)
            dd, w = oracle_mod.parabola(delta, MU, sigma, edge, w_formula=0, clamp_neg_d=0)
            if d2 < 1e-250:      # both derivatives underflow in double: w underflows too
                assert w < 1e-200
                continue
            assert 2 * w == pytest.approx(d2, rel=1e-9), (delta, edge)
            assert 2 * w * (delta - dd) == pytest.approx(d1, rel=1e-9), (delta, edge)
            dp, wp = oracle_mod.parabola(delta, MU, sigma, edge, w_formula=1, clamp_neg_d=0)
            assert 2 * wp * (delta - dp) == pytest.approx(d1, rel=1e-9), (delta, edge)
            assert wp >= w > 0   # the printed form adds c1 h^2, negligible when h underflows


def test_parabola_limits(oracle_mod):
    L2 = math.log(2)
    sigma = 0.8
    # far edge, u -> +inf: with h - u = 1/u - 2/u^3 + O(u^-5) (Mills ratio expansion),
    # d+ = mu - 2 sigma/u + O(u^-3) and w+ -> 1/(2 ln2 sigma^2) (derived reading)
    for u in (30.0, 200.0):
        dd, w = oracle_mod.parabola(MU + u * sigma, MU, sigma, True, clamp_neg_d=0)
        assert dd == pytest.approx(MU - 2 * sigma / u, abs=20 * sigma / u ** 3)
        assert w == pytest.approx(1 / (2 * L2 * sigma ** 2), rel=3 / u ** 2)
    # close non-edge, u -> -inf: mirror image, d- = mu + 2 sigma/|u| + O(|u|^-3)
    for u in (-30.0, -100.0):
        dd, w = oracle_mod.parabola(MU + u * sigma, MU, sigma, False, clamp_neg_d=0)
        assert dd == pytest.approx(MU + 2 * sigma / -u, abs=20 * sigma / u ** 2 / -u)
    # negative d+ for a close edge with a wide sigmoid, clamped to 0
    dd, _ = oracle_mod.parabola(0.1, MU, 1.0, True, clamp_neg_d=0)
    assert dd == pytest.approx(-0.5400, abs=1e-3)
    dd, _ = oracle_mod.parabola(0.1, MU, 1.0, True, clamp_neg_d=1)
    assert dd == 0.0


# ---------------------------------------------------------------------------
# Eq. 3: the update is a scaled gradient step on the frozen-pair surrogate
# ---------------------------------------------------------------------------
def test_eq3_gradient_identity(oracle_mod, sbm_small):
    """y_i - z_i x_i = -1/2 dL/dx_i with L = sum of dl over the epoch's pairs
    (all edges once, every sampled non-edge once, symmetric updates)."""
    rp, ci = sbm_small
    n = len(rp) - 1
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.5, 1.5, size=(n, 3))
    sigma, k, seed, ep = 0.6, 4, 1234, 7
    r = oracle_mod.epoch(rp, ci, x, sigma, ep, seed, k, clamp_neg_d=0, symmetric=1)
    samples = r["samples"]
    h = 1e-6
    for i in range(0, n, 7):
        for c in range(3):
            xp = x.copy(); xp[i, c] += h
            xm = x.copy(); xm[i, c] -= h
            g = (oracle_mod.surrogate_L(rp, ci, xp, sigma, samples)
                 - oracle_mod.surrogate_L(rp, ci, xm, sigma, samples)) / (2 * h)
            assert r["delta"][i, c] == pytest.approx(-0.5 * g, rel=2e-6, abs=1e-8), (i, c)
    # the update itself: x_new = y / z
    np.testing.assert_allclose(r["x_new"], r["y"] / r["z"][:, None], rtol=1e-15)


def test_edge_list_form_equals_csr_form(oracle_mod, sbm_small):
    """Fig. 4 walks the edge list and updates both endpoints; the per-vertex
    CSR sweep reaches every edge from both rows.  Same sums up to order."""
    rp, ci = sbm_small
    x = np.random.default_rng(1).normal(size=(len(rp) - 1, 2))
    for wf in (0, 1):
        y1, z1 = oracle_mod.edge_terms(rp, ci, x, 0.9, w_formula=wf, form="edgelist")
        y2, z2 = oracle_mod.edge_terms(rp, ci, x, 0.9, w_formula=wf, form="csr")
        np.testing.assert_allclose(y1, y2, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(z1, z2, rtol=1e-12)


def test_zmin_guard_keeps_isolated_far_vertex(oracle_mod):
    # vertex 2 is isolated and far from everyone: all its non-edge weights underflow
    rp = np.array([0, 1, 2, 2], dtype=np.int32)
    ci = np.array([1, 0], dtype=np.int32)
    x = np.array([[0.0, 0.0], [0.5, 0.0], [1e4, 1e4]])
    r = oracle_mod.epoch(rp, ci, x, 0.5, 0, 3, 2)
    assert r["z"][2] < 1e-30
    np.testing.assert_array_equal(r["x_new"][2], x[2])


# ---------------------------------------------------------------------------
# Sampling (Fig. 2 semantics)
# ---------------------------------------------------------------------------
def test_sampling_semantics(oracle_mod, sbm_small):
    rp, ci = sbm_small
    n = len(rp) - 1
    k, seed, ep, R = 6, 77, 4, 32
    s = oracle_mod.sample(rp, ci, ep, seed, k, max_retries=R)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    adj = [set(ci[rp[i]:rp[i + 1]].tolist()) for i in range(n)]
    rejected = 0
    for i in range(n):
        for t in range(k):
            # replay the candidate sequence from the (pinned) Philox words
            got = -1
            for a in range(R):
                r = int(oracle_mod.philox4x32_10([i, ep, t >> 2, 0x0B000000 | a], key)[t & 3])
                g = (r * n) >> 32
                if g != i and g not in adj[i]:
                    got = g
                    break
                rejected += 1
            assert s[i, t] == got
            assert got == -1 or (got != i and got not in adj[i])
    r = oracle_mod.epoch(rp, ci, np.zeros((n, 2)), 1.0, ep, seed, k)
    assert r["rejected"] == rejected
    np.testing.assert_array_equal(r["samples"], s)


def test_sampling_exhaustion_on_complete_row(oracle_mod):
    # star centre adjacent to everyone: every draw is an edge or itself
    n = 9
    rows = [list(range(1, n))] + [[0] for _ in range(1, n)]
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    ci = np.array(sum(rows, []), dtype=np.int32)
    r = oracle_mod.epoch(rp, ci, np.random.default_rng(0).normal(size=(n, 2)), 1.0, 0, 5, 3,
                         max_retries=8)
    assert (r["samples"][0] == -1).all()
    assert r["exhausted"] >= 3


# ---------------------------------------------------------------------------
# Slope optimisation (Sec. III.F)
# ---------------------------------------------------------------------------
def _epoch_hist(oracle_mod, sbm_1000, x_scale=1.0, sigma=1.0):
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    x = oracle_mod.init_positions(len(rp) - 1, 2, seed=5).astype(np.float64) * x_scale
    r = oracle_mod.epoch(rp, ci, x, sigma, 0, 5, 5)
    return r["hist_e"], r["hist_n"]


def test_dpe_dsigma_is_the_derivative(oracle_mod, sbm_1000):
    he, hn = _epoch_hist(oracle_mod, sbm_1000, x_scale=2.0)
    for s in (0.05, 0.4, 1.0, 3.0):
        h = s * 1e-6
        fd = (oracle_mod.hist_pe(he, hn, 12.0, MU, s + h) - oracle_mod.hist_pe(he, hn, 12.0, MU, s - h)) / (2 * h)
        assert oracle_mod.dpe_dsigma(he, hn, 12.0, MU, s) == pytest.approx(fd, rel=1e-6)


def test_sigma_fit_minimises_histogram_entropy(oracle_mod, sbm_1000):
    from scipy.optimize import minimize_scalar
    for scale in (1.0, 2.0, 4.0):
        he, hn = _epoch_hist(oracle_mod, sbm_1000, x_scale=scale)
        s = oracle_mod.sigma_fit(he, hn)
        res = minimize_scalar(lambda t: oracle_mod.hist_pe(he, hn, 12.0, MU, math.exp(t)),
                              bounds=(math.log(1e-3), math.log(1e3)), method="bounded",
                              options=dict(xatol=1e-10))
        assert s == pytest.approx(math.exp(res.x), rel=1e-4)


def test_sigma_fit_separable_goes_to_bracket_floor(oracle_mod):
    # edges all at 0.5, non-edges all at 3.0: entropy falls as sigma -> 0 (Sec. II.B: PE -> 0)
    B = 1024
    he = np.zeros(B); hn = np.zeros(B)
    he[int(0.5 / (12.0 / B))] = 100
    hn[int(3.0 / (12.0 / B))] = 5000
    s = oracle_mod.sigma_fit(he, hn)
    # any sigma whose entropy underflows to zero is a minimiser; the fit must reach one
    assert oracle_mod.hist_pe(he, hn, 12.0, MU, s) < 1e-100
    assert s < 0.05


# ---------------------------------------------------------------------------
# Eq. 2: predictive entropy
# ---------------------------------------------------------------------------
def test_loss_exact_against_scipy(oracle_mod, sbm_small):
    from scipy.special import log_ndtr
    rp, ci = sbm_small
    n = len(rp) - 1
    x = np.random.default_rng(3).normal(size=(n, 2))
    sigma = 0.7
    adj = np.zeros((n, n), dtype=bool)
    for i in range(n):
        adj[i, ci[rp[i]:rp[i + 1]]] = True
    iu = np.triu_indices(n, 1)
    dist = np.linalg.norm(x[iu[0]] - x[iu[1]], axis=1)
    u = (dist - MU) / sigma
    # s+ = Q(u) = Phi(-u), s- = Phi(u)
    dl = np.where(adj[iu], -log_ndtr(-u), -log_ndtr(u)) / math.log(2)
    ref = dl.sum() / (n * (n - 1) / 2)
    assert oracle_mod.loss_exact(rp, ci, x, sigma) == pytest.approx(ref, rel=1e-12)


def test_exact_dpe_dsigma_is_the_derivative(oracle_mod, sbm_small):
    """The exact dPE/dsigma against central differences of the exact Eq. 2
    (a different code path: orc_loss_exact sums dl directly)."""
    rp, ci = sbm_small
    n = len(rp) - 1
    N = n * (n - 1) / 2
    x = np.random.default_rng(8).normal(size=(n, 3)) * 1.3
    for sigma in (0.3, 0.9, 2.5):
        h = 1e-5 * sigma
        fd = (oracle_mod.loss_exact(rp, ci, x, sigma + h) - oracle_mod.loss_exact(rp, ci, x, sigma - h)) / (2 * h)
        assert oracle_mod.dpe_dsigma_exact(rp, ci, x, sigma) / N == pytest.approx(fd, rel=1e-6, abs=1e-12)


def test_exact_sigma_fit_minimises_eq2(oracle_mod, sbm_small):
    """The exact slope is a minimum of the exact Eq. 2 (mu fixed), and it is
    close to the slope fitted on fine distance histograms of the same pairs."""
    rp, ci = sbm_small
    n = len(rp) - 1
    x = np.random.default_rng(9).normal(size=(n, 2))
    s = oracle_mod.sigma_fit_exact(rp, ci, x)
    pe = oracle_mod.loss_exact(rp, ci, x, s)
    for f in (0.98, 0.995, 1.005, 1.02):
        assert oracle_mod.loss_exact(rp, ci, x, s * f) >= pe
    assert abs(oracle_mod.dpe_dsigma_exact(rp, ci, x, s)) < 1e-6 * abs(oracle_mod.dpe_dsigma_exact(rp, ci, x, 2 * s))
    # all pairs binned into 8192 bins on [0, 12): the histogram fit lands within a bin width or so
    adj = np.zeros((n, n), dtype=bool)
    for i in range(n):
        adj[i, ci[rp[i]:rp[i + 1]]] = True
    iu = np.triu_indices(n, 1)
    dist = np.linalg.norm(x[iu[0]] - x[iu[1]], axis=1)
    B = 8192
    b = np.minimum((dist / (12.0 / B)).astype(int), B - 1)
    he = np.bincount(b[adj[iu]], minlength=B).astype(float)
    hn = np.bincount(b[~adj[iu]], minlength=B).astype(float)
    assert oracle_mod.sigma_fit(he, hn, 12.0, MU) == pytest.approx(s, rel=2e-3)


def test_sampled_loss_is_unbiased(oracle_mod, sbm_small):
    rp, ci = sbm_small
    n = len(rp) - 1
    x = np.random.default_rng(4).normal(size=(n, 2))
    exact = oracle_mod.loss_exact(rp, ci, x, 0.8)
    est = np.array([oracle_mod.loss_sampled(rp, ci, x, 0.8, ep, 21, 4) for ep in range(400)])
    se = est.std(ddof=1) / math.sqrt(len(est))
    assert abs(est.mean() - exact) < 3.5 * se + 1e-12


def test_planted_embedding_entropy_vanishes(oracle_mod):
    # two cliques far apart: edges at distance ~0, non-edges at distance 10
    n = 12
    rows = [[j for j in range(6) if j != i] if i < 6 else [j for j in range(6, 12) if j != i] for i in range(n)]
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    ci = np.array(sum(rows, []), dtype=np.int32)
    x = np.zeros((n, 2)); x[6:, 0] = 10.0
    x[:, 1] = np.arange(n) % 6 * 1e-3
    pes = [oracle_mod.loss_exact(rp, ci, x, s) for s in (1.0, 0.3, 0.1)]
    assert pes[0] > pes[1] > pes[2] and pes[2] < 1e-6


def test_histograms_count_pairs(oracle_mod, sbm_1000):
    """Sec. III.F histograms: every undirected edge once (weight 1); sampled
    non-edges weighted so that their total is the number of non-edges."""
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    n = len(rp) - 1
    m = len(ci) // 2
    x = oracle_mod.init_positions(n, 2, seed=9).astype(np.float64) * 3.0
    r = oracle_mod.epoch(rp, ci, x, 0.8, 2, 9, 5)
    assert r["exhausted"] == 0
    assert r["hist_e"].sum() == m
    assert r["hist_n"].sum() == pytest.approx(n * (n - 1) / 2 - m, rel=1e-12)
    rows = np.repeat(np.arange(n), np.diff(rp))
    up = ci > rows
    de = np.linalg.norm(x[rows[up]] - x[ci[up]], axis=1)
    ref, _ = np.histogram(np.minimum(de, 12.0 - 1e-9), bins=1024, range=(0.0, 12.0))
    np.testing.assert_array_equal(r["hist_e"], ref)


# ---------------------------------------------------------------------------
# Block sampling (representation-learning form)
# ---------------------------------------------------------------------------
def test_block_sampling_semantics(oracle_mod, sbm_small):
    """Every vertex of a tile meets the tile's partners; pairs with the vertex
    itself or a neighbour are masked (not redrawn); the weights of the
    unmasked pairs add up to the number of non-edges; the gradient identity
    of Eq. 3 holds for the block pairs as for any pair list."""
    rp, ci = sbm_small
    n = len(rp) - 1
    T, P, seed, ep = 16, 12, 91, 3
    adj = [set(ci[rp[i]:rp[i + 1]].tolist()) for i in range(n)]
    x = np.random.default_rng(8).normal(size=(n, 2)) * 1.3
    r = oracle_mod.epoch(rp, ci, x, 0.8, ep, seed, k=5, block_partners=P, tile_vertices=T, clamp_neg_d=0)
    parts = r["partners"]
    assert parts.shape == ((n + T - 1) // T, P)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    masked = 0
    samples = np.full((n, P), -1, dtype=np.int32)
    for tile in range(parts.shape[0]):
        for p in range(P):
            word = int(oracle_mod.philox4x32_10([tile, ep, p >> 2, 0x0D000000], key)[p & 3])
            assert parts[tile, p] == (word * n) >> 32
        for i in range(tile * T, min(n, (tile + 1) * T)):
            for p in range(P):
                g = int(parts[tile, p])
                if g == i or g in adj[i]:
                    masked += 1
                else:
                    samples[i, p] = g
    assert r["rejected"] == masked and r["accepted"] == n * P - masked
    assert r["hist_n"].sum() == pytest.approx(n * (n - 1) / 2 - len(ci) // 2, rel=1e-12)
    # the per-vertex sample lists reproduce the epoch's sums through the identity
    h = 1e-6
    for i in range(0, n, 11):
        for c in range(2):
            xp = x.copy(); xp[i, c] += h
            xm = x.copy(); xm[i, c] -= h
            g = (oracle_mod.surrogate_L(rp, ci, xp, 0.8, samples)
                 - oracle_mod.surrogate_L(rp, ci, xm, 0.8, samples)) / (2 * h)
            assert r["delta"][i, c] == pytest.approx(-0.5 * g, rel=2e-6, abs=1e-8)


def test_per_slot_sampling_semantics(oracle_mod, sbm_small):
    """Sec. III.C's policy: one sample per CSR slot, anchored at the slot's
    row (so vertex i gets deg(i) samples), redrawn while it hits the anchor or
    an edge.  Checked: the draws follow the stated counter layout, every
    accepted sample is a non-edge of its anchor, the weights add up to the
    number of non-edges, k plays no part, and the epoch's sums obey the
    gradient identity of Eq. 3 for these pairs."""
    rp, ci = sbm_small
    n, nnz = len(rp) - 1, int(rp[-1])
    seed, ep = 4242, 5
    adj = [set(ci[rp[i]:rp[i + 1]].tolist()) for i in range(n)]
    x = np.random.default_rng(12).normal(size=(n, 2)) * 1.2
    r = oracle_mod.epoch(rp, ci, x, 0.8, ep, seed, k=3, per_slot=1, clamp_neg_d=0)
    smp = r["samples"]
    assert smp.shape == (nnz,)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    rejected = 0
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            got = -1
            for a in range(32):
                word = int(oracle_mod.philox4x32_10([e >> 2, ep, 0, 0x0C000000 | a], key)[e & 3])
                g = (word * n) >> 32
                if g != i and g not in adj[i]:
                    got = g
                    break
                rejected += 1
            assert smp[e] == got
            if got >= 0:
                assert got != i and got not in adj[i]
    assert r["rejected"] == rejected and r["accepted"] == int((smp >= 0).sum())
    if r["exhausted"] == 0:
        assert r["hist_n"].sum() == pytest.approx(n * (n - 1) / 2 - nnz // 2, rel=1e-12)
    # k plays no part in the per-slot policy
    r7 = oracle_mod.epoch(rp, ci, x, 0.8, ep, seed, k=7, per_slot=1, clamp_neg_d=0)
    np.testing.assert_array_equal(r7["samples"], smp)
    np.testing.assert_allclose(r7["delta"], r["delta"], rtol=0, atol=0)
    # gradient identity with the per-vertex lists of these samples
    maxdeg = int(np.diff(rp).max())
    lists = np.full((n, maxdeg), -1, dtype=np.int32)
    for i in range(n):
        lists[i, : rp[i + 1] - rp[i]] = smp[rp[i]:rp[i + 1]]
    h = 1e-6
    for i in range(0, n, 9):
        for c in range(2):
            xp = x.copy(); xp[i, c] += h
            xm = x.copy(); xm[i, c] -= h
            g = (oracle_mod.surrogate_L(rp, ci, xp, 0.8, lists)
                 - oracle_mod.surrogate_L(rp, ci, xm, 0.8, lists)) / (2 * h)
            assert r["delta"][i, c] == pytest.approx(-0.5 * g, rel=2e-6, abs=1e-8)


def test_separate_histogram_pass(oracle_mod, sbm_small):
    """Sec. III.F's separate pass: every edge once with weight 1, non-edge
    weights adding up to the number of non-edges, samples that are non-edges
    of their anchors; a run with it refits sigma from the new positions."""
    rp, ci = sbm_small
    n, m = len(rp) - 1, len(ci) // 2
    x = np.random.default_rng(21).normal(size=(n, 2))
    he, hn = oracle_mod.hist_pass(rp, ci, x, 3, 77, 6)
    assert he.sum() == m
    assert hn.sum() == pytest.approx(n * (n - 1) / 2 - m, rel=1e-12)
    # the edge histogram is the binned edge distances at x
    iu = [(i, j) for i in range(n) for j in ci[rp[i]:rp[i + 1]] if j > i]
    dist = np.array([np.linalg.norm(x[i] - x[j]) for i, j in iu])
    np.testing.assert_array_equal(he, np.bincount(np.minimum((dist / (12.0 / 1024)).astype(int), 1023),
                                                  minlength=1024))
    x0 = oracle_mod.init_positions(n, 2, 5)
    xa, sa, _ = oracle_mod.run(rp, ci, x0, 1.0, 3, 5, 4, sigma_source=1)
    xb, sb, _ = oracle_mod.run(rp, ci, x0, 1.0, 3, 5, 4, sigma_source=0)
    assert sa != sb
    # the last refit of the sigma_source=1 run is the fit on the pass at the
    # positions after its last epoch (epoch index 2)
    xr, sr, _ = oracle_mod.run(rp, ci, x0, 1.0, 2, 5, 4, sigma_source=1)
    r = oracle_mod.epoch(rp, ci, xr, sr, 2, 5, 4)
    he2, hn2 = oracle_mod.hist_pass(rp, ci, r["x_new"], 2, 5, 4)
    assert oracle_mod.sigma_fit(he2, hn2, 12.0, MU) == pytest.approx(sa, rel=1e-12)


def test_bytemap_membership(oracle_mod, sbm_small):
    """Sec. III.C's lossy membership test.  The renaming is a bijection; with
    a map large enough that the low bits of (i' n + j') never collide the
    byte map is exact (the samples equal the exact test's); with a small map
    no edge is ever accepted, colliding non-edges are rejected, and those
    false positives are what the count reports."""
    rp, ci = sbm_small
    n = len(rp) - 1
    adj = [set(ci[rp[i]:rp[i + 1]].tolist()) for i in range(n)]
    for period in (0, 1, 7):
        _, (a, b) = oracle_mod.bytemap_addr(n, 33, period, 12, [[0, 1]])
        assert math.gcd(a, n) == 1 and 1 <= a < n and 0 <= b < n
        assert sorted((a * v + b) % n for v in range(n)) == list(range(n))
    x = np.random.default_rng(5).normal(size=(n, 2))
    exact = oracle_mod.epoch(rp, ci, x, 0.8, 4, 33, 6)
    big = oracle_mod.epoch(rp, ci, x, 0.8, 4, 33, 6, membership=1, bytemap_log2=20)
    np.testing.assert_array_equal(big["samples"], exact["samples"])
    assert big["false_pos"] == 0
    small = oracle_mod.epoch(rp, ci, x, 0.8, 4, 33, 6, membership=1, bytemap_log2=8)
    smp = small["samples"]
    assert small["false_pos"] > 0
    for i in range(n):
        for g in smp[i]:
            if g >= 0:
                assert g != i and g not in adj[i]
    # replay the draws: a draw is rejected when it is i, an edge, or a pair
    # whose address is marked by some edge; the collisions are the false positives
    pairs = [(i, j) for i in range(n) for j in adj[i]]
    marked = set(oracle_mod.bytemap_addr(n, 33, 0, 8, pairs)[0].tolist())
    key = [33, 0]
    fp = rej = 0
    for i in range(n):
        for t in range(6):
            for att in range(32):
                w = int(oracle_mod.philox4x32_10([i, 4, t >> 2, 0x0B000000 | att], key)[t & 3])
                g = (w * n) >> 32
                addr = int(oracle_mod.bytemap_addr(n, 33, 0, 8, [[i, g]])[0][0])
                if g != i and addr not in marked:
                    assert smp[i, t] == g
                    break
                rej += 1
                fp += int(g != i and g not in adj[i])
    assert small["rejected"] == rej and small["false_pos"] == fp
    # renaming every 2 epochs: epochs 4 and 5 share a renaming, epoch 6 does not
    r4 = oracle_mod.epoch(rp, ci, x, 0.8, 4, 33, 6, membership=1, bytemap_log2=8, rename_every=2)
    assert r4["false_pos"] != small["false_pos"] or not np.array_equal(r4["samples"], smp)
    _, ab2 = oracle_mod.bytemap_addr(n, 33, 2, 8, [[0, 1]])
    _, ab3 = oracle_mod.bytemap_addr(n, 33, 3, 8, [[0, 1]])
    assert ab2 != ab3


def _bytemap_addr_restated(n, w0, w1, log2_size, i, j):
    """Sec. III.C's address, restated with Python integers from its definition:
    the renaming pi(v) = (a v + b) mod n (a = 1 + w0 mod (n-1), stepped up,
    wrapping to 1, to the first value coprime to n; b = w1 mod n), then
    hash = ((pi(i) n + pi(j)) * 1103515245) mod 2^32, masked to the map's
    s = 2^log2_size bytes.  Every 32-bit step is reduced mod 2^32 explicitly."""
    a = 1 + (w0 % (n - 1))
    while math.gcd(a, n) != 1:
        a = 1 if a + 1 >= n else a + 1
    b = w1 % n
    pi, pj = (a * i + b) % n, (a * j + b) % n
    t = (pi * n) % (1 << 32)
    t = (t + pj) % (1 << 32)
    t = (t * 1103515245) % (1 << 32)
    return t & ((1 << log2_size) - 1), (a, b)


@pytest.mark.parametrize("n", [1000, 70001, 131072, 1000003])
def test_bytemap_address_restated(oracle_mod, n):
    """The oracle's byte-map address equals its definition (Sec. III.C)
    restated here with Python integers, for graphs where pi(i) n + pi(j)
    stays below 2^32 (n = 1000) and where it wraps (n > 65536): operands in
    the other order, the map size s in place of s - 1, or a renaming other
    than the affine one fails.  The renaming's words come from the Philox
    function, which is pinned against cuRAND separately."""
    seed, rng = 0x1234ABCD, np.random.default_rng(n)
    for period, log2 in ((0, 12), (3, 20), (11, 30)):
        w0, w1 = (int(v) for v in oracle_mod.philox4x32_10([period, 0, 0, 0x09000000],
                                                          [seed & 0xFFFFFFFF, seed >> 32])[:2])
        pairs = rng.integers(0, n, size=(400, 2)).astype(np.int32)
        pairs[:4] = [[0, 0], [n - 1, n - 1], [0, n - 1], [n - 1, 0]]
        got, ab = oracle_mod.bytemap_addr(n, seed, period, log2, pairs)
        want = [_bytemap_addr_restated(n, w0, w1, log2, int(i), int(j)) for i, j in pairs]
        assert tuple(ab) == want[0][1]
        np.testing.assert_array_equal(got, np.array([w for w, _ in want], dtype=np.uint32))
        if n > 65536:
            a, b = want[0][1]
            big = [((a * int(i) + b) % n) * n + (a * int(j) + b) % n for i, j in pairs]
            assert max(big) >= 1 << 32, "the 32-bit wrap of pi(i) n + pi(j) is exercised"


@pytest.mark.parametrize("form", [dict(k=5), dict(k=5, symmetric=0), dict(k=3, per_slot=1),
                                  dict(k=0, block_partners=64, tile_vertices=128),
                                  dict(k=0, block_partners=16, tile_vertices=128, symmetric=0)],
                         ids=["per-vertex", "per-vertex-anchor-only", "per-slot", "block", "block-anchor-only"])
def test_vertex_terms_equal_whole_epoch(oracle_mod, sbm_1000, form):
    """Eq. 3 for chosen vertices alone (the full-size checks' reference)
    gives each chosen vertex the sums the whole epoch gives it: its edges,
    the non-edges sampled at it, and (symmetric) the non-edges whose sampled
    partner it is.  A dropped or doubled pair, a partner term sent to the
    anchor, or a mask missed changes y, z or the term sizes of some vertex."""
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    n = len(rp) - 1
    x = np.random.default_rng(31).normal(size=(n, 3)) * 1.1
    kw = dict(form)
    k = kw.pop("k")
    full = oracle_mod.epoch(rp, ci, x, 0.9, 6, 777, k, **kw)
    rng = np.random.default_rng(5)
    query = np.concatenate([[0, n - 1, int(np.argmax(np.diff(rp)))],
                            rng.choice(np.arange(1, n - 1), 60, replace=False)])
    query = np.unique(query)
    part = oracle_mod.vertex_terms(rp, ci, x, 0.9, 6, 777, k, query, **kw)
    np.testing.assert_allclose(part["y"], full["y"][query], rtol=1e-10, atol=1e-12 * float(np.abs(full["y"]).max()))
    np.testing.assert_allclose(part["z"], full["z"][query], rtol=1e-12)
    np.testing.assert_allclose(part["abs_terms"], full["abs_terms"][query], rtol=1e-12)
    np.testing.assert_allclose(part["delta"], full["delta"][query], rtol=0,
                               atol=1e-10 * float(full["abs_terms"].max()))
    np.testing.assert_allclose(part["x_new"], full["x_new"][query], rtol=1e-10, atol=1e-12)
    with pytest.raises(ValueError):
        oracle_mod.vertex_terms(rp, ci, x, 0.9, 6, 777, k, [3, 3], **kw)


def test_run_resumes_and_refits_on_cadence(oracle_mod, sbm_small):
    """Fig. 4 iterated: a run of 6 epochs equals 4 epochs then 2 more resumed
    from the reached state (the epoch counter keys the draws, so a wrong
    counter on resume changes the samples); sigma stays at sigma0 with
    sigma_every = 0 and is refitted only after every sigma_every-th epoch
    (Sec. III.F's fixed cadence)."""
    rp, ci = sbm_small
    n = len(rp) - 1
    x0 = oracle_mod.init_positions(n, 2, 99).astype(np.float64)
    x6, s6, st6 = oracle_mod.run(rp, ci, x0, 1.0, 6, 99, 4)
    x4, s4, st4 = oracle_mod.run(rp, ci, x0, 1.0, 4, 99, 4)
    x6b, s6b, st2 = oracle_mod.run(rp, ci, x4, s4, 2, 99, 4, epoch0=4)
    np.testing.assert_array_equal(x6b, x6)
    assert s6b == s6
    assert st4["accepted"] + st2["accepted"] == st6["accepted"]
    # resuming with the wrong epoch counter draws other samples
    x6c, _, _ = oracle_mod.run(rp, ci, x4, s4, 2, 99, 4, epoch0=0)
    assert np.abs(x6c - x6).max() > 1e-6
    # fixed sigma
    _, s_fixed, _ = oracle_mod.run(rp, ci, x0, 1.0, 3, 99, 4, sigma_every=0)
    assert s_fixed == 1.0
    # cadence 2: no refit after epoch 1, a refit after epoch 2
    _, s_one, _ = oracle_mod.run(rp, ci, x0, 1.0, 1, 99, 4, sigma_every=2)
    _, s_two, _ = oracle_mod.run(rp, ci, x0, 1.0, 2, 99, 4, sigma_every=2)
    assert s_one == 1.0 and s_two != 1.0


def test_golden_closed_forms_reproduce():
    """The stored closed-form values are what the committed generator computes
    from Eq. 4 / Eq. 5 with Python's math module (no oracle, no engine)."""
    import importlib.util
    path = os.path.join(HERE, "golden", "make_parabola_closed_forms.py")
    spec = importlib.util.spec_from_file_location("make_parabola_closed_forms", path)
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    with open(os.path.join(HERE, "golden", "parabola_closed_forms.txt")) as f:
        assert f.read() == gen.text()


# ---------------------------------------------------------------------------
# Sec. III.C's LCG and Fig. 2's float trick (rng = 1)
# ---------------------------------------------------------------------------
def _lcg_vertex_restated(state, n):
    """Fig. 2's map in numpy FP32: mantissa bits of the state in [1, 2), times
    n minus n (one FP32 rounding each), rounded to nearest-even; n is vertex 0."""
    f = np.array([0x3F800000 | (state & 0x7FFFFF)], dtype=np.uint32).view(np.float32)[0]
    nf = np.float32(n)
    t = np.float32(f * nf)
    t = np.float32(t - nf)
    g = int(np.rint(t))
    return g - n if g >= n else g


def test_lcg_step_and_vertex_map(oracle_mod):
    """The generator is s -> 1103515245 s + 1 mod 2^32; the map sends mantissa
    0 to vertex 0, mantissa 2^22 (f = 1.5) to n/2 (ties to even for odd n),
    the largest mantissa (f = 2 - 2^-23) to n, read as 0, for n < 2^22."""
    s = 12345
    for _ in range(50):
        nxt = oracle_mod.lcg_next(s)
        assert nxt == (s * 1103515245 + 1) % (1 << 32)
        s = nxt
    assert oracle_mod.lcg_next(0xFFFFFFFF) == (0xFFFFFFFF * 1103515245 + 1) % (1 << 32)
    for n in (2, 7, 97, 1000, 65537, 1000000):
        assert oracle_mod.lcg_vertex(0xABC00000 & ~0x7FFFFF, n) == 0
        half = oracle_mod.lcg_vertex(0x00400000, n)
        assert half == (n // 2 if n % 2 == 0 or (n // 2) % 2 == 0 else n // 2 + 1)
        assert oracle_mod.lcg_vertex(0x007FFFFF, n) == 0
    rng = np.random.default_rng(8)
    for n in (3, 60, 1001, 131072, 2_000_003):
        for st in rng.integers(0, 1 << 32, 300, dtype=np.uint64).tolist():
            g = oracle_mod.lcg_vertex(st, n)
            assert 0 <= g < n and g == _lcg_vertex_restated(int(st), n)


def test_lcg_vertices_uniform(oracle_mod):
    n, draws = 97, 97 * 400
    counts = np.zeros(n)
    s = 2024
    for _ in range(draws):
        s = (s * 1103515245 + 1) % (1 << 32)
        counts[oracle_mod.lcg_vertex(s, n)] += 1
    chi2 = ((counts - draws / n) ** 2 / (draws / n)).sum()
    from scipy.stats import chi2 as chi2d
    assert chi2d.sf(chi2, n - 1) > 1e-4


@pytest.mark.parametrize("per_slot", [0, 1])
def test_lcg_samples_replayed(oracle_mod, sbm_small, per_slot):
    """rng = 1: every sample slot's state is seeded from its Philox word
    ((i, epoch, t>>2, 0x08000000) word t&3; per-slot policy (e>>2, epoch, 0,
    0x07000000) word e&3) and advanced once per attempt (Fig. 2: the state
    moves before each draw); a draw of the anchor itself or a neighbour is
    redrawn.  Replayed here attempt by attempt from the definition."""
    rp, ci = sbm_small
    n = len(rp) - 1
    adj = [set(ci[rp[i]:rp[i + 1]].tolist()) for i in range(n)]
    seed, epoch, k = 4242, 3, 6
    key = [seed & 0xFFFFFFFF, seed >> 32]
    x = np.random.default_rng(2).normal(size=(n, 2))
    r = oracle_mod.epoch(rp, ci, x, 0.9, epoch, seed, k, per_slot=per_slot, rng=1)
    ref = oracle_mod.epoch(rp, ci, x, 0.9, epoch, seed, k, per_slot=per_slot, rng=0)
    assert not np.array_equal(r["samples"], ref["samples"])
    rej = 0
    slots = [(i, rp[i] + t if per_slot else t) for i in range(n)
             for t in (range(rp[i + 1] - rp[i]) if per_slot else range(k))]
    got = r["samples"].reshape(-1)
    for i, t in slots:
        if per_slot:
            st = int(oracle_mod.philox4x32_10([t >> 2, epoch, 0, 0x07000000], key)[t & 3])
            out = got[t]
        else:
            st = int(oracle_mod.philox4x32_10([i, epoch, t >> 2, 0x08000000], key)[t & 3])
            out = got[i * k + t]
        want = -1
        for _ in range(32):
            st = (st * 1103515245 + 1) % (1 << 32)
            g = _lcg_vertex_restated(st, n)
            if g != i and g not in adj[i]:
                want = g
                break
            rej += 1
        assert out == want, (i, t)
    assert r["rejected"] == rej


@pytest.mark.parametrize("form", [dict(k=5), dict(k=3, per_slot=1), dict(k=0, block_partners=64),
                                  dict(k=4, symmetric=0)], ids=["per-vertex", "per-slot", "block", "anchor-only"])
def test_epoch_over_anchor_ranges_adds_up(oracle_mod, sbm_1000, form):
    """Sec. III.E splits Eq. 3's numerators and denominators over workers:
    the terms of the anchors of each range of a partition, added up, are the
    whole epoch's sums, histograms, counts and samples (ranges on tiles of
    128 in the block form)."""
    rp, ci = sbm_1000["row_ptr"], sbm_1000["col_idx"]
    x = np.random.default_rng(12).normal(size=(1000, 3))
    kw = dict(form)
    k = kw.pop("k")
    full = oracle_mod.epoch(rp, ci, x, 0.9, 4, 77, k, **kw)
    cuts = [0, 256, 640, 1000] if kw.get("block_partners") else [0, 333, 334, 801, 1000]
    parts = [oracle_mod.epoch(rp, ci, x, 0.9, 4, 77, k, anchors=(a, b), **kw) for a, b in zip(cuts, cuts[1:])]
    for f in ("y", "z", "hist_e", "hist_n"):
        tot = sum(p[f] for p in parts)
        np.testing.assert_allclose(tot, full[f], rtol=1e-12, atol=1e-12 * float(np.abs(full[f]).max()))
    for f in ("accepted", "rejected", "exhausted"):
        assert sum(p[f] for p in parts) == full[f]
    with pytest.raises(ValueError):
        oracle_mod.epoch(rp, ci, x, 0.9, 4, 77, k, anchors=(10, 5), **kw)
