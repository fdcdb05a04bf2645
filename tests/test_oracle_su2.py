"""Pins of the SU(2) oracle (Eqs. (2)-(7), heat-bath, Sec. 2.4) against what the
mathematics and physics fix: Pauli algebra, the exact heat-bath density,
the Wilson action, gauge invariance, strong and weak coupling, Haar moments."""
import math

import numpy as np
import pytest
from scipy import stats

from conftest import binned_mean_err
from oracle import exact

SIGMA = [np.array([[0, 1], [1, 0]], dtype=complex),
         np.array([[0, -1j], [1j, 0]], dtype=complex),
         np.array([[1, 0], [0, -1]], dtype=complex)]


def quat_to_matrix(q):
    """Eq. (4) with explicit Pauli matrices."""
    return q[0] * np.eye(2) + 1j * sum(q[k + 1] * SIGMA[k] for k in range(3))


def matrix_to_quat(U):
    return np.array([np.trace(U).real / 2] + [(np.trace(SIGMA[k] @ U) / 2j).real for k in range(3)])


def random_unit_quats(rng, n):
    g = rng.normal(size=(n, 4))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def test_product_matches_pauli_algebra(orc):
    rng = np.random.default_rng(1)
    for a, b in zip(random_unit_quats(rng, 50), random_unit_quats(rng, 50)):
        want = matrix_to_quat(quat_to_matrix(a) @ quat_to_matrix(b))
        np.testing.assert_allclose(orc.su2_mul(a, b), want, atol=1e-14)
        # and the matrix is in SU(2)
        M = quat_to_matrix(a)
        np.testing.assert_allclose(M @ M.conj().T, np.eye(2), atol=1e-14)
        assert abs(np.linalg.det(M) - 1) < 1e-14


@pytest.mark.parametrize("alpha", [0.01, 0.5, 2.0, 5.0, 10.0])
def test_heatbath_a0_distribution(orc, alpha):
    """KS test of the combined Kennedy-Pendleton + Creutz sampler against the
    exact density sqrt(1-a^2) e^{alpha a}, and of each stage on its own (a draw
    accepted by either stage must follow the density); mean = I2/I1."""
    n = 200_000
    a0, tries = orc.su2_sample_a0(alpha, seed=99, n=n)
    assert (tries != orc.HB_FAILED).all()
    cdf = lambda x: exact.heatbath_cdf_vec(x, alpha)
    assert stats.kstest(a0, cdf).pvalue > 1e-4
    for sel in (tries < 8, tries >= 8):
        if sel.sum() > 2000:
            assert stats.kstest(a0[sel], cdf).pvalue > 1e-4
    want = exact.heatbath_mean(alpha)
    assert abs(a0.mean() - want) < 4.5 * a0.std() / math.sqrt(n)


def test_heatbath_small_alpha_uses_fallback(orc):
    """Kennedy-Pendleton is inefficient at small alpha, so the Creutz stage must
    carry a visible share there and almost none at large alpha."""
    _, t_small = orc.su2_sample_a0(0.3, seed=5, n=20000)
    _, t_large = orc.su2_sample_a0(8.0, seed=5, n=20000)
    assert (t_small >= 8).mean() > 0.02
    assert (t_large >= 8).mean() < 1e-3


def test_staple_reproduces_action_difference(orc):
    """Replacing one link U by U' changes the Wilson action (Eq. (2), computed
    from the plaquettes of Eq. (3)) by -beta/2 [Re Tr(U' W^+) - Re Tr(U W^+)],
    W the staple of Eq. (6); Re Tr(U W^+) = 2 (U . W) for quaternions.
    Asymmetric extents pin the direction bookkeeping."""
    L = [6, 4, 8, 4]
    beta = 2.3
    rng = np.random.default_rng(3)
    ns = int(np.prod(L))
    q = random_unit_quats(rng, ns * 4).reshape(ns, 4, 4).copy()
    S0 = orc.su2_action(q, L, beta)
    for _ in range(12):
        s = int(rng.integers(ns))
        mu = int(rng.integers(4))
        W = orc.su2_staple(q, L, s, mu)
        new = random_unit_quats(rng, 1)[0]
        q2 = q.copy()
        q2[s, mu] = new
        dS = orc.su2_action(q2, L, beta) - S0
        want = -beta / 2 * (2 * np.dot(new, W) - 2 * np.dot(q[s, mu], W))
        assert dS == pytest.approx(want, abs=1e-9)


def test_plaquette_gauge_invariance(orc):
    L = [4, 4, 6, 4]
    rng = np.random.default_rng(4)
    ns = int(np.prod(L))
    q = random_unit_quats(rng, ns * 4).reshape(ns, 4, 4).copy()
    P0 = orc.su2_plaquette(q, L)
    g = random_unit_quats(rng, ns)

    def coords(s):
        x1 = s % L[1]; s //= L[1]
        x2 = s % L[2]; s //= L[2]
        x3 = s % L[3]; s //= L[3]
        return [s, x1, x2, x3]

    def index(x):
        return x[1] + L[1] * (x[2] + L[2] * (x[3] + L[3] * x[0]))

    def dag(v):
        return np.array([v[0], -v[1], -v[2], -v[3]])

    qg = np.empty_like(q)
    for s in range(ns):
        for mu in range(4):
            x = coords(s)
            x[mu] = (x[mu] + 1) % L[mu]
            qg[s, mu] = orc.su2_mul(orc.su2_mul(g[s], q[s, mu]), dag(g[index(x)]))
    np.testing.assert_allclose(orc.su2_plaquette(qg, L), P0, atol=1e-13)
    assert abs(P0[0]) < 0.05  # random links


def test_cold_and_hot_start(orc):
    L = [8, 8, 8, 8]
    cold = orc.su2_init(L, seed=1, hot=False)
    np.testing.assert_allclose(orc.su2_plaquette(cold, L), [1, 1, 1], atol=0)
    hot = orc.su2_init(L, seed=1, chain=0, hot=True).reshape(-1, 4)
    np.testing.assert_allclose(np.linalg.norm(hot, axis=1), 1.0, atol=1e-14)
    n = hot.shape[0]
    # Haar measure: <a_k> = 0, <a_k^2> = 1/4 for each component
    for k in range(4):
        assert abs(hot[:, k].mean()) < 4.5 * 0.5 / math.sqrt(n)
        assert abs((hot[:, k] ** 2).mean() - 0.25) < 4.5 * 0.25 / math.sqrt(n)
    assert abs(orc.su2_plaquette(hot.reshape(-1, 4, 4), L)[0]) < 0.02


def test_heatbath_update_pit_uniform(orc):
    """Probability-integral transform of the whole link update.  The links of
    the last phase of a sweep (even sites, mu = 3) see, at update time, the
    staple computed from the final configuration; X = U V^+ (V = W/k) must have
    a0 distributed with density sqrt(1-a^2) e^{beta k a}, i.e. CDF(a0) uniform,
    and a uniformly distributed direction."""
    L = [8, 8, 8, 8]
    beta = 2.0
    q = orc.su2_init(L, seed=12, chain=0, hot=True)
    orc.su2_sweep(q, L, beta, seed=12, chain=0, sweep=0)
    pit, dirs = [], []
    ns = int(np.prod(L))
    for s in range(ns):
        x = [s % 8, (s // 8) % 8, (s // 64) % 8, s // 512]
        if sum(x) % 2 != 0:
            continue
        W = orc.su2_staple(q, L, s, 3)
        k = np.linalg.norm(W)
        V = W / k
        Vd = np.array([V[0], -V[1], -V[2], -V[3]])
        X = orc.su2_mul(q[s, 3], Vd)
        pit.append(exact.heatbath_cdf_vec(np.array([X[0]]), beta * k)[0])
        dirs.append(X[1:] / np.linalg.norm(X[1:]))
    pit = np.array(pit)
    dirs = np.array(dirs)
    assert stats.kstest(pit, "uniform").pvalue > 1e-4
    n = len(dirs)
    assert np.all(np.abs(dirs.mean(axis=0)) < 4.5 / math.sqrt(3 * n))
    assert stats.kstest(dirs[:, 2], stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-4


def test_unit_norm_after_sweeps(orc):
    L = [4, 6, 4, 4]
    q = orc.su2_init(L, seed=2, hot=True)
    for k in range(5):
        orc.su2_sweep(q, L, 2.3, 2, 0, k)
    np.testing.assert_allclose(np.linalg.norm(q.reshape(-1, 4), axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("beta", [0.1, 0.2])
def test_strong_coupling_plaquette(orc, beta):
    """At small beta the plaquette is the single-plaquette value I2(beta)/I1(beta)
    (~ beta/4) up to corrections of order (beta/4)^5 from closed surfaces."""
    L = [4, 4, 4, 4]
    q = orc.su2_init(L, seed=7, hot=True)
    P = []
    for k in range(2300):
        orc.su2_sweep(q, L, beta, 7, 0, k)
        if k >= 300:
            P.append(orc.su2_plaquette(q, L)[0])
    mean, err = binned_mean_err(P, 20)
    want = exact.strong_coupling_plaquette(beta)
    assert abs(mean - want) < 4.5 * err + 1e-4, (mean, want, err)


def test_weak_coupling_plaquette(orc):
    """Leading perturbative order for SU(2): 1 - <P> = 3/(4 beta) (+ O(1/beta^2))."""
    L = [4, 4, 4, 4]
    beta = 40.0
    q = orc.su2_init(L, seed=8, hot=False)
    P = []
    for k in range(200):
        orc.su2_sweep(q, L, beta, 8, 0, k)
        if k >= 50:
            P.append(orc.su2_plaquette(q, L)[0])
    one_minus = 1 - np.mean(P)
    assert one_minus == pytest.approx(3 / (4 * beta), rel=0.1)


def test_forced_tries_protocol(orc):
    """Following one's own decisions is a no-op with nothing counted; forcing a
    try that contradicts a decision far from its threshold is counted as bad."""
    L = [4, 4, 4, 4]
    q0 = orc.su2_init(L, seed=3, hot=True)
    a = q0.copy()
    tries, fails, near, bad = orc.su2_sweep(a, L, 2.0, 3, 0, 0)
    assert fails == 0 and near == 0 and bad == 0
    b = q0.copy()
    _, _, near, bad = orc.su2_sweep(b, L, 2.0, 3, 0, 0, forced_tries=tries)
    assert near == 0 and bad == 0
    np.testing.assert_array_equal(a, b)
    planted = tries.copy()
    s = int(np.argmax(planted[:, 0] == 0))
    planted[s, 0] = 1  # claim try 0 was rejected
    c = q0.copy()
    _, _, near, bad = orc.su2_sweep(c, L, 2.0, 3, 0, 0, forced_tries=planted)
    assert bad >= 1


# ------------------------------------------------------------------ overrelaxation
def _gauge_transform(orc, q, L, g):
    """U_mu(x) -> g(x) U_mu(x) g(x + mu)^dag."""
    ns = int(np.prod(L))

    def shifted(s, mu):
        x1 = s % L[1]; r = s // L[1]
        x2 = r % L[2]; r //= L[2]
        x3 = r % L[3]; x0 = r // L[3]
        x = [x0, x1, x2, x3]
        x[mu] = (x[mu] + 1) % L[mu]
        return x[1] + L[1] * (x[2] + L[2] * (x[3] + L[3] * x[0]))

    out = np.empty_like(q)
    for s in range(ns):
        for mu in range(4):
            gd = g[shifted(s, mu)] * np.array([1, -1, -1, -1])
            out[s, mu] = orc.su2_mul(orc.su2_mul(g[s], q[s, mu]), gd)
    return out


@pytest.mark.parametrize("L", [[4, 4, 4, 4], [2, 4, 6, 4]])
def test_overrelaxation_preserves_the_action(orc, L):
    """Each reflection keeps Re Tr(U W^dag), the only part of the Wilson action
    (Eq. (2)) that depends on the link, so a whole overrelaxation sweep leaves
    the action unchanged while moving every link."""
    q = orc.su2_init(L, seed=11, hot=True)
    q0 = q.copy()
    S0 = orc.su2_action(q, L, 2.3)
    for _ in range(3):
        orc.su2_overrelax(q, L)
        assert abs(orc.su2_action(q, L, 2.3) - S0) < 1e-11 * abs(S0)
    assert np.abs(q - q0).max() > 0.5  # it is not the identity
    np.testing.assert_allclose(np.linalg.norm(q.reshape(-1, 4), axis=1), 1.0, atol=1e-14)


def test_overrelaxation_is_gauge_covariant(orc):
    """Reflecting then gauge transforming equals gauge transforming then
    reflecting: fixes the orientation of the staple and of the reflection
    (V^dag U^dag V^dag, say, keeps neither the action nor this)."""
    L = [4, 4, 2, 4]
    rng = np.random.default_rng(12)
    ns = int(np.prod(L))
    q = random_unit_quats(rng, ns * 4).reshape(ns, 4, 4).copy()
    g = random_unit_quats(rng, ns)
    a = q.copy()
    orc.su2_overrelax(a, L)
    a = _gauge_transform(orc, a, L, g)
    b = _gauge_transform(orc, q, L, g)
    orc.su2_overrelax(b, L)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_heatbath_with_overrelaxation_strong_coupling(orc):
    """One heat-bath plus two overrelaxation sweeps per step still samples the
    Wilson measure: the strong-coupling plaquette I2(b)/I1(b) at b = 0.2."""
    L = [4, 4, 4, 4]
    beta = 0.2
    q = orc.su2_init(L, seed=13, hot=True)
    P = []
    for k in range(1800):
        orc.su2_sweep(q, L, beta, 13, 0, k)
        orc.su2_overrelax(q, L)
        orc.su2_overrelax(q, L)
        if k >= 300:
            P.append(orc.su2_plaquette(q, L)[0])
    mean, err = binned_mean_err(P, 20)
    want = exact.strong_coupling_plaquette(beta)
    assert abs(mean - want) < 4.5 * err + 1e-4, (mean, want, err)


# ------------------------------------------------------------------ Polyakov loop
def test_polyakov_cold_and_uniform_rotation(orc):
    """Cold links give 1; U_0 = exp(i theta sigma_3) everywhere gives the closed
    form cos(L_0 theta) (the loop winds L_0 times)."""
    for L in ([4, 4, 4, 4], [6, 2, 4, 2]):
        q = orc.su2_init(L, seed=1, hot=False)
        assert orc.su2_polyakov(q, L) == 1.0
        theta = 0.37
        q[:, 0] = [math.cos(theta), 0.0, 0.0, math.sin(theta)]
        assert orc.su2_polyakov(q, L) == pytest.approx(math.cos(L[0] * theta), abs=1e-14)


def test_polyakov_gauge_invariance_and_centre_flip(orc):
    """Invariant under U_mu(x) -> g(x) U_mu(x) g(x+mu)^dag (which telescopes only
    for the time-ordered product), odd under flipping the sign of every U_0 on
    one time slice (a centre transformation)."""
    L = [4, 2, 4, 2]
    rng = np.random.default_rng(14)
    ns = int(np.prod(L))
    q = random_unit_quats(rng, ns * 4).reshape(ns, 4, 4).copy()
    p0 = orc.su2_polyakov(q, L)
    g = random_unit_quats(rng, ns)
    assert orc.su2_polyakov(_gauge_transform(orc, q, L, g), L) == pytest.approx(p0, abs=1e-13)
    nspace = L[1] * L[2] * L[3]
    flipped = q.copy()
    flipped[2 * nspace:3 * nspace, 0] *= -1  # time slice x0 = 2
    assert orc.su2_polyakov(flipped, L) == pytest.approx(-p0, abs=1e-14)
    assert abs(p0) > 1e-4  # not trivially zero
