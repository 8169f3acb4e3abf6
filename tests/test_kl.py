"""The KL divergence of 2D normals used by the UT / EWA accuracy study, against closed forms."""
import math

import numpy as np

from paper_2412_12507_gb300.kl_study import gauss_kl


def test_kl_of_identical_normals_is_zero():
    m = np.array([[1.0, -2.0]])
    C = np.array([[[2.0, 0.3], [0.3, 1.0]]])
    assert abs(gauss_kl(m, C, m, C)[0]) < 1e-14


def test_kl_scaled_covariance_and_shift_closed_form():
    """KL(N(0, I) || N(mu, s I)) in 2D = (2/s + |mu|^2 / s - 2 + 2 ln s) / 2."""
    for s, mu in ((2.0, (0.0, 0.0)), (0.5, (0.3, -0.4)), (3.0, (1.0, 2.0))):
        m1 = np.array([mu])
        k = gauss_kl(np.zeros((1, 2)), np.eye(2)[None], m1, s * np.eye(2)[None])[0]
        ref = 0.5 * (2 / s + (mu[0] ** 2 + mu[1] ** 2) / s - 2 + 2 * math.log(s))
        assert abs(k - ref) < 1e-12


def test_kl_matches_monte_carlo_estimate():
    """E_P[log p - log q] by sampling agrees with the closed form."""
    rng = np.random.default_rng(0)
    m0, m1 = np.array([0.2, -0.1]), np.array([0.5, 0.3])
    C0 = np.array([[1.0, 0.4], [0.4, 0.8]])
    C1 = np.array([[1.5, -0.2], [-0.2, 0.6]])
    x = rng.multivariate_normal(m0, C0, 400_000)

    def logpdf(x, m, C):
        d = x - m
        return -0.5 * np.einsum("ni,ij,nj->n", d, np.linalg.inv(C), d) - 0.5 * np.log(np.linalg.det(2 * np.pi * C))

    mc = np.mean(logpdf(x, m0, C0) - logpdf(x, m1, C1))
    k = gauss_kl(m0[None], C0[None], m1[None], C1[None])[0]
    assert abs(mc - k) < 5e-3
