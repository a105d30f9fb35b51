"""Pins of the oracle's fermion determinant and Green's function against results that
do not come from the oracle itself: closed forms (lambda = 0, space-uniform field,
static staggered field, atomic limit), brute-force LU of the NL x NL block matrix,
and exact symmetries of the determinant."""
import numpy as np
import pytest

from oracle import HolsteinParams
from oracle.fermion import block_matrix, fermion_logdet, slice_matrix, udt_chain
from oracle.lattice import dispersion, exp_hopping, hopping_matrix, staggered_sign
from oracle.weight import bose_log_weight, log_weight


def params(Lx=4, L=40, n_s=10, lam=1.0, t=1.0, mu=0.0, dtau=0.1, Ly=None):
    return HolsteinParams(Lx, Ly or Lx, L, dtau=dtau, t=t, mu=mu, lam=lam, n_s=n_s)


def test_hopping_spectrum_is_band_dispersion():
    for Lx, Ly in ((4, 4), (6, 4), (2, 2), (3, 5)):
        K = hopping_matrix(Lx, Ly, 1.3, 0.2)
        eps, _, _ = dispersion(Lx, Ly, 1.3, 0.2)
        assert np.allclose(np.sort(np.linalg.eigvalsh(K)), np.sort(eps), atol=1e-12)
        assert np.allclose(K, K.T)


def test_exp_hopping_against_series():
    K = hopping_matrix(4, 4, 1.0, 0.0)
    A = -0.1 * K
    S = np.eye(16)
    term = np.eye(16)
    for n in range(1, 30):
        term = term @ A / n
        S = S + term
    assert np.abs(exp_hopping(4, 4, 1.0, 0.0, 0.1) - S).max() < 1e-14


@pytest.mark.parametrize("Lx,L,n_s", [(4, 40, 10), (4, 37, 8), (6, 60, 7), (8, 80, 10)])
def test_lambda_zero_closed_form(Lx, L, n_s):
    p = params(Lx, L, n_s, lam=0.0)
    eps, KX, KY = dispersion(Lx, Lx, p.t, p.mu)
    x = np.random.default_rng(0).normal(size=(p.N, L))
    lndet, sign, G = fermion_logdet(p, x)
    ref = np.sum(np.log1p(np.exp(-p.beta * eps)))
    assert sign == 1
    assert abs(lndet - ref) < 1e-10 * max(1.0, abs(ref))
    # G = (1 + e^{-beta K})^{-1}: G_ij = (1/N) sum_k cos(k.(r_i - r_j)) f(eps_k)
    ix = np.arange(p.N) % Lx
    iy = np.arange(p.N) // Lx
    dx = ix[:, None] - ix[None, :]
    dy = iy[:, None] - iy[None, :]
    f = 1.0 / (1.0 + np.exp(-p.beta * eps))
    Gref = np.einsum("k,ijk->ij", f, np.cos(KX[None, None, :] * dx[:, :, None]
                                            + KY[None, None, :] * dy[:, :, None])) / p.N
    assert np.abs(G - Gref).max() < 1e-11


def test_large_beta_lambda_zero():
    p = params(16, 160, 8, lam=0.0)
    eps, _, _ = dispersion(16, 16, 1.0, 0.0)
    x = np.zeros((256, 160))
    lndet, _, _ = fermion_logdet(p, x, want_G=False)
    ref = np.sum(np.log1p(np.exp(-p.beta * eps)))
    assert abs(lndet - ref) < 1e-9 * abs(ref)


def test_uniform_field_closed_form():
    p = params(4, 30, 7)
    c = np.random.default_rng(1).normal(size=30)
    x = np.repeat(c[None, :], p.N, axis=0)
    eps, _, _ = dispersion(4, 4, 1.0, 0.0)
    ref = np.sum(np.log1p(np.exp(-p.dtau * p.lam * c.sum() - p.beta * eps)))
    lndet, sign, _ = fermion_logdet(p, x)
    assert sign == 1 and abs(lndet - ref) < 1e-10 * abs(ref)


@pytest.mark.parametrize("Lx,L,m", [(4, 40, 0.8), (6, 120, 1.3), (12, 120, 0.8)])
def test_static_staggered_field_closed_form(Lx, L, m):
    # A field m (-1)^(ix+iy) couples k and k+(pi,pi); each 2x2 block has slice matrix
    # exp(-dtau lam m sigma_x) diag(e^{-dtau eps}, e^{+dtau eps}) of unit determinant and
    # trace 2 cosh(dtau lam m) cosh(dtau eps) = 2 cosh(theta), so
    # ln det = sum_k ln(2 cosh(L theta_k / 2)).
    p = params(Lx, L, 10)
    s = staggered_sign(Lx, Lx)
    x = np.repeat((m * s)[:, None], L, axis=1)
    eps, _, _ = dispersion(Lx, Lx, 1.0, 0.0)
    theta = np.arccosh(np.cosh(p.dtau * p.lam * m) * np.cosh(p.dtau * eps))
    ref = np.sum(np.log(2.0 * np.cosh(L * theta / 2.0)))
    lndet, sign, _ = fermion_logdet(p, x, want_G=False)
    assert sign == 1 and abs(lndet - ref) < 1e-10 * abs(ref)


def test_atomic_limit_closed_form():
    p = params(4, 40, 10, t=0.0)
    x = np.random.default_rng(2).normal(size=(16, 40))
    ref = np.sum(np.log1p(np.exp(-p.dtau * p.lam * x.sum(axis=1))))
    lndet, sign, G = fermion_logdet(p, x)
    assert abs(lndet - ref) < 1e-12 * abs(ref)
    assert np.allclose(G, np.diag(1.0 / (1.0 + np.exp(-p.dtau * p.lam * x.sum(axis=1)))), atol=1e-14)


@pytest.mark.parametrize("Lx,L,n_s,scale", [(4, 40, 10, 1.0), (4, 24, 5, 2.5), (2, 12, 4, 1.0), (6, 16, 3, 1.5)])
def test_brute_force_block_matrix(Lx, L, n_s, scale):
    p = params(Lx, L, n_s)
    E = exp_hopping(Lx, Lx, p.t, p.mu, p.dtau)
    x = scale * np.random.default_rng(Lx * L).normal(size=(p.N, L))
    O = block_matrix(E, x, p.dtau, p.lam)
    so, lo = np.linalg.slogdet(O)
    lndet, sign, G = fermion_logdet(p, x, E=E)
    assert abs(lndet - lo) < 1e-10 * max(1, abs(lo))
    assert sign == int(so)
    Oinv = np.linalg.inv(O)
    assert np.abs(G - Oinv[-p.N:, -p.N:]).max() < 1e-10


def test_small_beta_direct_product():
    p = params(4, 8, 3)
    E = exp_hopping(4, 4, p.t, p.mu, p.dtau)
    x = np.random.default_rng(3).normal(size=(16, 8))
    P = np.eye(16)
    for l in range(8):
        P = slice_matrix(E, x[:, l], p.dtau, p.lam) @ P
    s, ld = np.linalg.slogdet(np.eye(16) + P)
    lndet, sign, G = fermion_logdet(p, x, E=E)
    assert abs(ld - lndet) < 1e-12 * abs(ld) and sign == int(s)
    assert np.abs(G - np.linalg.inv(np.eye(16) + P)).max() < 1e-13
    U, D, T = udt_chain(E, x, p.dtau, p.lam, p.n_s)
    assert np.abs(U @ np.diag(D) @ T - P).max() < 1e-12 * np.abs(P).max()


def test_negative_sign_possible_and_matches_brute_force():
    # A strongly fluctuating field can make one species' determinant negative. The
    # regime (dtau = 1, 3-sigma fields) is ill-conditioned for both methods, hence the
    # looser magnitude tolerance; the sign must agree exactly.
    rng = np.random.default_rng(11)
    found = False
    for trial in range(100):
        p = params(2, 6, 1, lam=1.0, dtau=1.0)
        E = exp_hopping(2, 2, 1.0, 0.0, 1.0)
        x = 3.0 * rng.normal(size=(4, 6))
        so, lo = np.linalg.slogdet(block_matrix(E, x, p.dtau, p.lam))
        lndet, sign, _ = fermion_logdet(p, x, E=E)
        assert sign == int(so) and abs(lndet - lo) < 1e-7 * max(1, abs(lo))
        found |= sign < 0
    assert found


def test_particle_hole_identity():
    # Half filling on a bipartite lattice: ln det(I+B(-x)) = ln det(I+B(x)) + dtau lam sum x,
    # G(-x) = I - S G(x)^T S, so ln w is even in x.
    for Lx, L, n_s in ((4, 40, 10), (6, 48, 8)):
        p = params(Lx, L, n_s)
        x = np.random.default_rng(Lx).normal(size=(p.N, L))
        l1, s1, G1 = fermion_logdet(p, x)
        l2, s2, G2 = fermion_logdet(p, -x)
        assert abs(l2 - (l1 + p.dtau * p.lam * x.sum())) < 1e-10 * abs(l1)
        S = np.diag(staggered_sign(Lx, Lx))
        assert np.abs(G2 - (np.eye(p.N) - S @ G1.T @ S)).max() < 1e-10
        assert abs(log_weight(p, x)[0] - log_weight(p, -x)[0]) < 1e-9 * abs(log_weight(p, x)[0])


def test_translation_and_time_symmetries():
    p = params(4, 40, 10)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(16, 40))
    l0, _, _ = fermion_logdet(p, x, want_G=False)
    X = x.reshape(4, 4, 40)
    shifted = np.roll(np.roll(X, 1, axis=1), 2, axis=0).reshape(16, 40)
    assert abs(fermion_logdet(p, shifted, want_G=False)[0] - l0) < 1e-11 * abs(l0)
    assert abs(fermion_logdet(p, np.roll(x, 7, axis=1), want_G=False)[0] - l0) < 1e-11 * abs(l0)
    assert abs(fermion_logdet(p, x[:, ::-1].copy(), want_G=False)[0] - l0) < 1e-11 * abs(l0)


def test_bose_log_weight_by_loops():
    p = params(2, 3, 3, lam=0.7)
    x = np.random.default_rng(9).normal(size=(4, 3))
    ref = 0.0
    for i in range(4):
        for l in range(3):
            ref += p.dtau * p.lam * x[i, l]
            ref -= p.dtau * (p.omega0 ** 2 / 2 * x[i, l] ** 2
                             + (x[i, (l + 1) % 3] - x[i, l]) ** 2 / (2 * p.dtau ** 2))
    assert abs(bose_log_weight(p, x) - ref) < 1e-13
