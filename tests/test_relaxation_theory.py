"""The over-relaxation of the FP32 Newton correction's red updates, checked
on a model problem (numpy, no GPU).

The sweeps update black from red, then red from black, and relax every red
update: e_r <- e_r + omega (e_GS - e_r).  On a red-black (two-cyclic)
matrix with Jacobi eigenvalues +-mu the red error is then multiplied per
sweep by 1 - omega (1 - mu^2); over mu^2 in [0, rho^2] the largest factor
is smallest at omega = 2/(2 - rho^2), where it equals rho^2/(2 - rho^2),
about half of Gauss-Seidel's rho^2.  The model is the implicit diffusion
operator (1 + 4 s) e - s (sum of the four neighbours) on an n x n grid
with zero boundary values, whose Jacobi radius is
rho = 4 s cos(pi/(n + 1))/(1 + 4 s)."""
import numpy as np
import pytest


def _sweep(e, s, omega):
    """One black-then-red sweep of the homogeneous problem (the error)."""
    n = e.shape[0]
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    red = (I + J) % 2 == 0
    d = 1.0 + 4.0 * s

    def nb(x):
        y = np.zeros_like(x)
        y[1:, :] += x[:-1, :]
        y[:-1, :] += x[1:, :]
        y[:, 1:] += x[:, :-1]
        y[:, :-1] += x[:, 1:]
        return y

    e = e.copy()
    e[~red] = (s * nb(e) / d)[~red]                 # black from red
    gs = s * nb(e) / d                              # red from the new black
    e[red] = e[red] + omega * (gs[red] - e[red])
    return e


def _rate(s, omega, n=24, sweeps=400, seed=3):
    """Asymptotic contraction per sweep (ratio of norms over the last 100)."""
    e = np.random.default_rng(seed).standard_normal((n, n))
    hist = []
    for _ in range(sweeps):
        e = _sweep(e, s, omega)
        hist.append(np.linalg.norm(e))
        e /= hist[-1]                               # keep it representable
    return float(np.exp(np.mean(np.log(hist[-100:]))))


def _theory(rho2, omega):
    return max(abs(1.0 - omega), abs(1.0 - omega * (1.0 - rho2)))


@pytest.mark.parametrize("s", [0.0819, 0.25])
def test_red_over_relaxation_factor(s):
    n = 24
    rho = 4.0 * s * np.cos(np.pi / (n + 1)) / (1.0 + 4.0 * s)
    rho2 = rho * rho
    opt = 2.0 / (2.0 - rho2)
    for omega in (1.0, 0.5 * (1.0 + opt), opt, 1.0 + 1.5 * (opt - 1.0)):
        assert _rate(s, omega, n) == pytest.approx(_theory(rho2, omega), rel=0.03), omega
    # Gauss-Seidel's factor is rho^2; the optimum's about half of it
    assert _rate(s, 1.0, n) == pytest.approx(rho2, rel=0.03)
    assert _rate(s, opt, n) == pytest.approx(rho2 / (2.0 - rho2), rel=0.05)
    # and no omega on a fine scan does better
    best = min(_rate(s, w, n) for w in np.linspace(1.0, 1.0 + 3.0 * (opt - 1.0), 13))
    assert _rate(s, opt, n) <= best * 1.05
